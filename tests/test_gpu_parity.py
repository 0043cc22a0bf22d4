"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: neighbour lists bit-exact; FP64 right-hand side, filter, RK steps and dt
within 1e-12 relative L2 of the oracle given identical weights; GPU-built FP64
weights within a conditioning-scaled bound; FP32 results within the rounding
budget derived in test_gpu_fp32.py.
"""
import math

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2102_02019_gb300 as lb
    return lb


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


class Case:
    """A node set with its oracle stencil, oracle weights and GPU-built data."""

    def __init__(self, lb, ns, rows_for_weights=None):
        self.ns = ns
        self.xy = _dev(ns.xy)
        self.h = _dev(ns.h)
        self.s = _dev(ns.s)
        self.row_ptr, self.col = lb.build_stencils(self.xy, self.h, ns.Lx, ns.Ly)
        self.rp_o, self.col_o = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
        self.gw = lb.build_weights(self.xy, self.h, self.s, ns.Lx, ns.Ly, self.row_ptr, self.col, ns.m)
        self.ow = oracle.build_weights(ns.xy, ns.h, ns.s, self.rp_o, self.col_o, ns.m, ns.Lx, ns.Ly,
                                       want_cond=True)


@pytest.fixture(scope="module")
def c1(lb):
    # 64 x 64 jittered lattice, m = 4, h/s = 1.7 (the small Taylor-Green workload)
    return Case(lb, li.tgv_lattice(64, m=4, h_over_s=1.7, jitter=0.3, seed=0))


@pytest.fixture(scope="module")
def ragged(lb):
    # non-square ragged lattice, m = 6
    return Case(lb, li.tgv_lattice(37, 29, m=6, h_over_s=2.2, jitter=0.3, seed=5))


# ---------------------------------------------------------------- stencils

def test_stencils_bit_exact_small(c1, ragged):
    for c in (c1, ragged):
        assert np.array_equal(c.row_ptr.cpu().numpy(), c.rp_o)
        assert np.array_equal(c.col.cpu().numpy(), c.col_o)


@pytest.mark.parametrize("case", ["varh", "nonperiodic", "tiny", "wide_h"])
def test_stencils_bit_exact_edge_cases(lb, case):
    if case == "varh":
        ns = li.tgv_lattice(40, 33, m=4, jitter=0.3, seed=8)
        ns.h = ns.h * np.random.default_rng(3).uniform(0.7, 1.6, size=ns.N)
        per = (True, True)
    elif case == "nonperiodic":
        ns = li.tgv_lattice(30, 30, m=4, jitter=0.3, seed=9)
        per = (False, False)
    elif case == "tiny":
        ns = li.tgv_lattice(3, 2, m=2, jitter=0.3, seed=10)
        per = (True, True)
    else:  # stencil wider than half the box: every cell visited once
        ns = li.tgv_lattice(6, 5, m=2, h_over_s=2.9, jitter=0.3, seed=11)
        per = (True, True)
    xy, h = _dev(ns.xy), _dev(ns.h)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly, periodic=per)
    rp_o, col_o = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=per)
    assert np.array_equal(rp.cpu().numpy(), rp_o)
    assert np.array_equal(col.cpu().numpy(), col_o)


def test_stencil_points_exactly_on_the_radius(lb):
    # offsets of exactly 2h (representable) must be included, as in the oracle
    xy = np.array([[0.25, 0.25], [0.5, 0.25], [0.25, 0.5], [0.75, 0.75], [0.0, 0.25]])
    h = np.full(5, 0.125)
    rp, col = lb.build_stencils(_dev(xy), _dev(h), 1.0, 1.0)
    rp_o, col_o = oracle.neighbours(xy, h, 1.0, 1.0)
    assert np.array_equal(rp.cpu().numpy(), rp_o) and np.array_equal(col.cpu().numpy(), col_o)
    assert 1 in col_o[rp_o[0]:rp_o[1]] and 2 in col_o[rp_o[0]:rp_o[1]]


def test_stencil_capacity_and_invalid_input(lb):
    ns = li.tgv_lattice(16, m=4, seed=1)
    xy, h = _dev(ns.xy), _dev(ns.h)
    import ctypes
    N = ns.N
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    small = torch.full((10,), -7, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64(0)
    st = torch.cuda.current_stream().cuda_stream
    rc = lb.lib.labfm_build_stencils(xy.data_ptr(), h.data_ptr(), N, ns.Lx, ns.Ly, 3, rp.data_ptr(),
                                     small.data_ptr(), 10, ctypes.byref(nnz), st)
    assert rc == 4 and nnz.value > 10
    assert torch.all(small == -7)  # nothing written past the capacity check
    bad = ns.xy.copy()
    bad[5, 0] = 1.5  # outside the box
    with pytest.raises(lb.LabfmError) as ei:
        lb.build_stencils(_dev(bad), h, ns.Lx, ns.Ly)
    assert ei.value.status == 1


def test_malformed_csr_is_refused_before_any_kernel_uses_it(lb):
    # a caller's CSR is checked when a plan, weights, an optimisation or a modal
    # response is asked for it: row_ptr[0] = 0, non-decreasing, row_ptr[N] = nnz,
    # columns in [0, N).  Every buffer here has the declared size; only its
    # contents are wrong, so the checks read nothing out of bounds
    ns = li.tgv_lattice(16, m=4, seed=1)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4)
    N, nnz = ns.N, col.numel()
    cases = {}
    c = col.clone()
    c[nnz // 2] = N
    cases["column >= N"] = (rp, c)
    c = col.clone()
    c[3] = -1
    cases["negative column"] = (rp, c)
    r = rp.clone()
    r[7], r[8] = r[8], r[7].clone() + 1
    cases["row_ptr decreases"] = (r, col)
    r = rp.clone()
    r[0] = 1
    cases["row_ptr[0] != 0"] = (r, col)
    for name, (r, c) in cases.items():
        with pytest.raises(lb.LabfmError) as ei:
            lb.Plan(r, c, wb["w"], wb["kappa"], s, dtype=torch.float32)
        assert ei.value.status == 1, name
        with pytest.raises(lb.LabfmError) as ei:
            lb.build_weights(xy, h, s, ns.Lx, ns.Ly, r, c, 4)
        assert ei.value.status == 1, name
        with pytest.raises(lb.LabfmError):
            lb.modal_response(xy, s, ns.Lx, ns.Ly, r, c, wb["w"], nk=4)
        with pytest.raises(lb.LabfmError):
            lb.stencil_optimise(xy, h, s, ns.Lx, ns.Ly, r, c, 4, max_iter=1)
    # row_ptr[N] != nnz: the plan is given one column fewer than the rows cover
    with pytest.raises(lb.LabfmError) as ei:
        lb.Plan(rp, col[:-1], wb["w"][:, :-1], wb["kappa"], s, dtype=torch.float64)
    assert ei.value.status == 1 and "row_ptr[N]" in str(ei.value)
    # a batched plan names the instance
    inst = [dict(row_ptr=rp, col=col, w=wb["w"], kappa=wb["kappa"], s=s),
            dict(row_ptr=rp, col=cases["column >= N"][1], w=wb["w"], kappa=wb["kappa"], s=s)]
    with pytest.raises(lb.LabfmError) as ei:
        lb.Plan.batched(inst, dtype=torch.float32)
    assert ei.value.status == 1 and "instance 1" in str(ei.value)
    # the well-formed CSR still makes a plan that steps
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float32)
    Q = _dev(li.tgv_fields(ns.xy, 10.0), torch.float32)
    lb.rk_step(plan, Q, 1e-4, 2, lb.Phys(100.0, 0.005))
    assert bool(torch.isfinite(Q).all())
    plan.close()


# ---------------------------------------------------------------- weights

def _weight_errors(c):
    """Per node: max over operators of |w_gpu - w_oracle| / max_j |w_oracle| for that operator."""
    wg = c.gw["w"].cpu().numpy()
    wo = c.ow["w"]
    rp = c.rp_o
    N = len(rp) - 1
    err = np.zeros(N)
    for i in range(N):
        sl = slice(rp[i], rp[i + 1])
        scale = np.abs(wo[:, sl]).max(axis=1, keepdims=True)
        err[i] = (np.abs(wg[:, sl] - wo[:, sl]) / scale).max()
    return err


def test_weights_match_oracle_within_conditioning(c1, ragged):
    for c in (c1, ragged):
        n = oracle.n_unknowns(c.ns.m)
        assert int(c.gw["status"].abs().sum().item()) == 0
        err = _weight_errors(c)
        bound = np.maximum(50.0 * n * EPS64 * c.ow["cond1"], 1e-13)
        assert np.all(err <= bound), (err / bound).max()
        kg = c.gw["kappa"].cpu().numpy()
        ko = c.ow["kappa"]
        assert np.all(np.abs(kg - ko) <= np.abs(ko) * bound)
        # reproduction residual of eq. lsys, nondimensional
        assert float(c.gw["residual"].max().item()) < 1e-10 * max(1.0, 6.0 * (c.ns.m // 2))


@pytest.mark.parametrize("m,hs,nx", [(2, 1.2, 20), (8, 2.8, 24), (10, 3.3, 24)])
def test_weights_other_orders(lb, m, hs, nx):
    ns = li.tgv_lattice(nx, m=m, h_over_s=hs, jitter=0.3, seed=20 + m)
    c = Case(lb, ns)
    assert int(c.gw["status"].abs().sum().item()) == 0
    # operator outputs on smooth functions agree far inside the raw-weight bound
    wg = c.gw["w"].cpu().numpy()
    wo = c.ow["w"]
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    f = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.3 * np.cos(4 * np.pi * x)
    for d in range(5):
        lg = oracle.apply_op(f, wg[d], c.rp_o, c.col_o)
        lo = oracle.apply_op(f, wo[d], c.rp_o, c.col_o)
        scale = np.abs(lo).max()
        assert np.abs(lg - lo).max() <= 1e-7 * scale, (d, np.abs(lg - lo).max() / scale)
    err = _weight_errors(c)
    n = oracle.n_unknowns(m)
    bound = np.maximum(50.0 * n * EPS64 * c.ow["cond1"], 1e-13)
    assert np.all(err <= bound)


def test_weights_flag_nodes_with_too_few_neighbours(lb):
    ns = li.tgv_lattice(12, m=8, h_over_s=1.0, jitter=0.3, seed=3)  # ~12 neighbours < n = 44
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    with pytest.raises(lb.LabfmError) as ei:
        lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 8, check=True)
    assert ei.value.status == 5
    out = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 8)
    st = out["status"].cpu().numpy()
    assert np.all(st & lb.NODE_FEW_NEIGHBOURS)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n_side", [1, 5])
def test_empty_stencils_leave_the_state_unchanged(lb, dtype, n_side):
    # degenerate node sets: a single node, or stencils too small to hold a neighbour.
    # Every stencil is empty (nnz = 0), so every derivative and kappa are zero, the
    # right-hand side of eq. icns is zero and a time step (stages and filter) is the
    # identity, bit for bit, with the plain, the persistent and the prefetching kernels
    ns = li.tgv_lattice(n_side, m=2, h_over_s=0.2, jitter=0.0, seed=4)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    assert col.numel() == 0 and int(rp[-1].item()) == 0
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 2)
    assert np.all(wb["status"].cpu().numpy() & lb.NODE_FEW_NEIGHBOURS)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
    q0 = _dev(li.tgv_fields(ns.xy, 10.0), dtype)
    phys = lb.Phys(100.0, 0.005)
    assert float(lb.rhs(plan, q0, phys).abs().max().item()) == 0.0
    for persistent in (False, True):
        plan.set_persistent(persistent)
        Q = q0.clone()
        lb.rk_step(plan, Q, 1e-3, 3, phys)
        assert torch.equal(Q, q0), persistent
    plan.close()


# ---------------------------------------------------------------- right-hand side, FP64

def _plan(lb, c, w, kappa, dtype):
    return lb.Plan(c.row_ptr, c.col, _dev(w) if isinstance(w, np.ndarray) else w,
                   _dev(kappa) if isinstance(kappa, np.ndarray) else kappa, c.s, dtype=dtype)


def _rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("which", ["c1", "ragged"])
def test_rhs_fp64_matches_oracle(lb, c1, ragged, which):
    c = c1 if which == "c1" else ragged
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], torch.float64)
    q = li.perturbed_tgv_fields(c.ns.xy, 10.0, amplitude=0.05, kmax=4)
    phys = lb.Phys(c2=100.0, mu=0.005, gx=0.1, gy=-0.2)
    R = lb.rhs(plan, _dev(q), phys).cpu().numpy()
    Ro = oracle.rhs(q, c.ow["w"][:5], c.rp_o, c.col_o, 100.0, 0.005, (0.1, -0.2))
    assert np.all(_rel_l2(R, Ro) <= 1e-12), _rel_l2(R, Ro)
    # every launch shape gives the same result to rounding
    for g, b in ((4, 128), (16, 256), (32, 512)):
        plan.set_launch(g, b)
        R2 = lb.rhs(plan, _dev(q), phys).cpu().numpy()
        assert np.all(_rel_l2(R2, Ro) <= 1e-12)


def test_filter_fp64_matches_oracle(lb, c1):
    c = c1
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], torch.float64)
    q = li.perturbed_tgv_fields(c.ns.xy, 10.0, amplitude=0.1, kmax=8)
    F = lb.filter(plan, _dev(q)).cpu().numpy()
    Fo = oracle.filter_fields(q, c.ow["w"][5], c.ow["kappa"], c.rp_o, c.col_o)
    # compare the filter increments (the fields themselves agree trivially)
    assert np.all(_rel_l2(F - q, Fo - q) <= 1e-12), _rel_l2(F - q, Fo - q)


def test_stable_dt_matches_oracle(lb, c1):
    c = c1
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], torch.float64)
    q = li.tgv_fields(c.ns.xy, 10.0)
    for mu in (0.005, 2.0):
        dt = float(lb.stable_dt(plan, _dev(q), c.s, 10.0, mu).item())
        dto = oracle.stable_dt(q, c.ns.s, 10.0, mu)
        assert abs(dt - dto) <= 4 * EPS64 * dto


@pytest.mark.parametrize("nsteps", [1, 3])
def test_rk_step_fp64_matches_oracle(lb, c1, nsteps):
    c = c1
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], torch.float64)
    q0 = li.tgv_fields(c.ns.xy, 10.0)
    dt = oracle.stable_dt(q0, c.ns.s, 10.0, 0.005)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, nsteps, lb.Phys(100.0, 0.005))
    qo = q0
    for _ in range(nsteps):
        qo = oracle.time_step(qo, dt, c.ow["w"], c.ow["kappa"], c.rp_o, c.col_o, 100.0, 0.005)
    # compare the change over the steps, a stricter test than the state
    assert np.all(_rel_l2(Q.cpu().numpy() - q0, qo - q0) <= 1e-12)


def test_trajectory_fp64_100_steps(lb):
    # the small Taylor-Green workload geometry with the regular jitter of the
    # stable runs (+-0.1 s), 100 steps, GPU-built weights on both sides
    ns = li.tgv_lattice(64, m=4, h_over_s=1.7, jitter=0.1, seed=0)
    c = Case(lb, ns)
    wg = c.gw["w"].cpu().numpy()
    kg = c.gw["kappa"].cpu().numpy()
    plan = _plan(lb, c, c.gw["w"], c.gw["kappa"], torch.float64)
    q0 = li.tgv_fields(ns.xy, 10.0)
    dt = oracle.stable_dt(q0, ns.s, 10.0, 0.005)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 100, lb.Phys(100.0, 0.005))
    qo = q0
    for _ in range(100):
        qo = oracle.time_step(qo, dt, wg, kg, c.rp_o, c.col_o, 100.0, 0.005)
    assert np.all(_rel_l2(Q.cpu().numpy(), qo) <= 1e-12), _rel_l2(Q.cpu().numpy(), qo)
    assert np.all(_rel_l2(Q.cpu().numpy() - q0, qo - q0) <= 1e-10)


def test_trajectory_fp64_100_steps_configured_geometry_shifted(lb):
    # the small Taylor-Green workload as configured (64 x 64, +-0.3 s jitter, m = 4,
    # h/s = 1.7) after the paper's ten iterations of iterative shifting (Section 5):
    # 100 FP64 steps stay finite and match the oracle, GPU-built weights on both sides
    ns = li.tgv_lattice(64, m=4, h_over_s=1.7, jitter=0.3, seed=0, shift_iterations=10)
    c = Case(lb, ns)
    wg = c.gw["w"].cpu().numpy()
    kg = c.gw["kappa"].cpu().numpy()
    plan = _plan(lb, c, c.gw["w"], c.gw["kappa"], torch.float64)
    q0 = li.tgv_fields(ns.xy, 10.0)
    dt = oracle.stable_dt(q0, ns.s, 10.0, 0.005)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 100, lb.Phys(100.0, 0.005))
    qo = q0
    for _ in range(100):
        qo = oracle.time_step(qo, dt, wg, kg, c.rp_o, c.col_o, 100.0, 0.005)
    qg = Q.cpu().numpy()
    assert np.all(np.isfinite(qg)) and np.all(np.isfinite(qo))
    assert np.abs(qo[1:]).max() < 1.0  # decaying vortex, no growth
    assert np.all(_rel_l2(qg, qo) <= 1e-12), _rel_l2(qg, qo)
    assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-10)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_filter_launch_shapes(lb, c1, dtype):
    # the filter's own lanes per node and its persistent grid: the persistent grid
    # gives the same state bit for bit; other lane counts sum in another order.  FP64:
    # two steps to 1e-12; FP32: one step elementwise within the derived
    # step budget
    from tests.fp32_budget import step_bound
    c = c1
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], dtype)
    q0 = li.tgv_fields(c.ns.xy, 10.0)
    dt = oracle.stable_dt(q0, c.ns.s, 10.0, 0.005)
    phys = lb.Phys(100.0, 0.005)
    nsteps = 2 if dtype == torch.float64 else 1
    ref = _dev(q0, dtype)
    lb.rk_step(plan, ref, dt, nsteps, phys)
    qo = q0
    for _ in range(nsteps):
        qo = oracle.time_step(qo, dt, c.ow["w"], c.ow["kappa"], c.rp_o, c.col_o, 100.0, 0.005)
    if dtype == torch.float32:
        bound = step_bound(q0, qo, dt, c.ow["w"], c.ow["kappa"], c.rp_o, c.col_o, 100.0, 0.005)
    for fg in (2, 4, 8, 16, 32):
        states = []
        for fp in (False, True):
            plan.set_filter_launch(fg, fp)
            info = plan.info()
            assert info["filter_group"] == fg and info["filter_persistent"] == int(fp)
            Q = _dev(q0, dtype)
            lb.rk_step(plan, Q, dt, nsteps, phys)
            states.append(Q)
        assert torch.equal(states[0], states[1]), fg
        qg = states[0].double().cpu().numpy()
        if dtype == torch.float64:  # the change over the steps, as in the step tests
            assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-12), (fg, _rel_l2(qg - q0, qo - q0))
        else:
            ratio = np.abs(qg - qo) / np.where(bound > 0, bound, np.inf)
            assert ratio.max() <= 1.0, (fg, ratio.max())
        if fg == 4:  # the plan's own group: identical to the default launch
            assert torch.equal(states[0], ref)
    plan.set_filter_launch(0, False)
    with pytest.raises(lb.LabfmError):
        plan.set_filter_launch(3, False)


def test_zero_steps_and_bad_workspace(lb, c1):
    c = c1
    plan = _plan(lb, c, c.ow["w"], c.ow["kappa"], torch.float64)
    q0 = _dev(li.tgv_fields(c.ns.xy, 10.0))
    Q = q0.clone()
    lb.rk_step(plan, Q, 1e-3, 0, lb.Phys(100.0, 0.005))
    assert torch.equal(Q, q0)
    with pytest.raises(lb.LabfmError):
        lb.rk_step(plan, Q, 1e-3, 1, lb.Phys(100.0, 0.005),
                   work=torch.empty(16, dtype=torch.uint8, device="cuda"))


# ---------------------------------------------------------------- full-size workload, sampled

@pytest.fixture(scope="module")
def c2(lb):
    ns = li.tgv_lattice(512, m=8, h_over_s=2.8, jitter=0.3, seed=1)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, ns.m)
    rows = np.random.default_rng(0).choice(ns.N, size=96, replace=False)
    rows = np.unique(np.concatenate([[0, ns.N - 1], rows]))
    return dict(ns=ns, xy=xy, h=h, s=s, rp=rp, col=col, wb=wb, rows=rows)


def test_fullsize_stencil_rows_bit_exact(c2):
    ns = c2["ns"]
    rp = c2["rp"].cpu().numpy()
    col = c2["col"].cpu().numpy()
    for i in c2["rows"]:
        ref = oracle.neighbours_of(ns.xy, ns.h, int(i), ns.Lx, ns.Ly)
        assert np.array_equal(col[rp[i]:rp[i + 1]], ref)
    assert abs(rp[-1] / ns.N / (4 * math.pi * 2.8 ** 2) - 1) < 0.02


def test_fullsize_weights_sampled(c2):
    ns = c2["ns"]
    rows = c2["rows"]
    rp = c2["rp"].cpu().numpy()
    col = c2["col"].cpu().numpy()
    rp_r = np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])])
    col_r = np.concatenate([col[rp[i]:rp[i + 1]] for i in rows])
    ow = oracle.build_weights(ns.xy, ns.h, ns.s, rp_r, col_r, ns.m, ns.Lx, ns.Ly, rows=rows,
                              want_cond=True)
    wg = c2["wb"]["w"].cpu().numpy()
    assert int(c2["wb"]["status"].abs().sum().item()) == 0
    n = oracle.n_unknowns(ns.m)
    for k, i in enumerate(rows):
        a, b = rp[i], rp[i + 1]
        wo = ow["w"][:, rp_r[k]:rp_r[k + 1]]
        scale = np.abs(wo).max(axis=1, keepdims=True)
        err = (np.abs(wg[:, a:b] - wo) / scale).max()
        assert err <= max(50 * n * EPS64 * ow["cond1"][k], 1e-13)


def test_fullsize_rhs_fp64_sampled(lb, c2):
    ns = c2["ns"]
    plan = lb.Plan(c2["rp"], c2["col"], c2["wb"]["w"], c2["wb"]["kappa"], c2["s"], dtype=torch.float64)
    q = li.tgv_fields(ns.xy, 10.0)
    R = lb.rhs(plan, _dev(q), lb.Phys(100.0, 0.005)).cpu().numpy()
    rows = c2["rows"]
    rp = c2["rp"].cpu().numpy()
    col = c2["col"].cpu().numpy()
    wg = c2["wb"]["w"].cpu().numpy()
    # oracle RHS at the sampled rows with the same weights
    cnt = np.zeros(ns.N, dtype=np.int64)
    cnt[rows] = rp[rows + 1] - rp[rows]
    rps = np.concatenate([[0], np.cumsum(cnt)])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    Ro = oracle.rhs(q, wg[:5, idx], rps, col[idx], 100.0, 0.005)
    for f in range(3):
        err = np.abs(R[f][rows] - Ro[f][rows]).max() / np.abs(Ro[f][rows]).max()
        assert err <= 1e-12, (f, err)
    plan.close()


def test_fullsize_fp32_in_the_bench_launch_shape(lb, c2):
    # the headline path as bench.py times it: 4 lanes per node, 128-thread blocks, the
    # record prefetch on (the plan default for these rows).  The sampled FP32 RHS is held
    # to the FP32 budget against the oracle, and one full FP32 time step to the per-node
    # budget of test_gpu_fp32 against the FP64 step (which matches the oracle to 1e-12)
    from test_gpu_fp32 import U32, _deriv_bound, rhs_bound
    ns, rows = c2["ns"], c2["rows"]
    rp, col = c2["rp"].cpu().numpy(), c2["col"].cpu().numpy()
    w, kap = c2["wb"]["w"], c2["wb"]["kappa"]
    wg = w.cpu().numpy()
    q = li.tgv_fields(ns.xy, 10.0)
    phys = lb.Phys(100.0, 0.005)
    p32 = lb.Plan(c2["rp"], c2["col"], w, kap, c2["s"], dtype=torch.float32)
    p32.set_launch(4, 128)
    assert p32.info()["prefetch"] == 2
    cnt = np.zeros(ns.N, dtype=np.int64)
    cnt[rows] = rp[rows + 1] - rp[rows]
    rps = np.concatenate([[0], np.cumsum(cnt)])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    Ro = oracle.rhs(q, wg[:5, idx], rps, col[idx], 100.0, 0.005)
    B = rhs_bound(q, wg[:, idx], rps, col[idx], 100.0, 0.005)
    R = lb.rhs(p32, _dev(q, torch.float32), phys).double().cpu().numpy()
    ratio = np.abs(R[:, rows] - Ro[:, rows]) / B[:, rows]
    assert ratio.max() <= 1.0, ratio.max()
    # one step
    p64 = lb.Plan(c2["rp"], c2["col"], w, kap, c2["s"], dtype=torch.float64)
    dt = oracle.stable_dt(q, ns.s, 10.0, 0.005)
    Q64 = _dev(q)
    lb.rk_step(p64, Q64, dt, 1, phys)
    Q32 = _dev(q, torch.float32)
    lb.rk_step(p32, Q32, dt, 1, phys)
    q1 = Q64.cpu().numpy()
    got = Q32.double().cpu().numpy()
    Bfull = rhs_bound(q, wg, rp, col, 100.0, 0.005)
    bsum = sum(abs(float(b)) for b in oracle.RK_B)
    wf = wg[5] * np.repeat(kap.cpu().numpy(), np.diff(rp))
    ri = oracle.row_index(rp)
    for f in range(3):
        bf, _ = _deriv_bound(q1[f], wf, rp, col)
        # A: the per-node budget of the state before the filter (as in test_gpu_fp32);
        # the filter of Section 6, phi_i + kappa_i sum_j (phi_j - phi_i) w^hyp_ji,
        # carries the errors of node i and of its neighbours with weights |kappa_i
        # w^hyp_ji| (large at the few irregular stencils with an outsized kappa), and
        # adds its own rounding budget bf
        A = 8 * U32 * np.abs(q1[f]) + 2 * dt * bsum * Bfull[f]
        carried = np.bincount(ri, np.abs(wf) * (A[col] + A[ri]), minlength=ns.N)
        bound = A + carried + 2 * bf
        assert np.all(np.abs(got[f] - q1[f]) <= bound), (f, (np.abs(got[f] - q1[f]) / bound).max())
    p32.close()
    p64.close()
