"""Open boundaries on the GPU (Section 7.1: the outflow of eq. outflowL and the
inflow, both in LODI form) against the oracle, on a box bounded in x (inflow at
x = 0, outflow at x = L) and periodic in y: the boundary operator with the
"FD + 1D-LABFM" second derivatives at the boundary nodes, the right-hand side at
every node, whole time steps, the closed forms of the relaxation terms, and an
acoustic pulse that leaves through the outflow where a wall sends it back."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import boundary_oracle as bo
from oracle import core as oracle
from tests.conftest import golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
C, U0, MU = 20.0, 1.0, 1e-3


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


def _rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _sigma():
    return {k: float(v) for k, v in golden("nscbc.txt")}["sigma"]


class Box:
    """An open box with the oracle's operator and the GPU-built one; the left
    boundary an inflow at (U0, 0), the right one an outflow to p_inf = c^2 (or a
    wall, by ``right``)."""

    def __init__(self, lb, nx, ny, m=6, m_wall=4, jitter=0.05, seed=1, right=bo.OUTFLOW, u_in=U0, mach=U0 / C):
        self.ns = ns = li.open_box(nx, ny, m=m, jitter=jitter, seed=seed)
        self.columns, self.normals = li.channel_walls(ns)
        self.xy, self.h, self.s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
        self.gop = lb.build_wall_operator(self.xy, self.h, self.s, ns.Lx, ns.Ly, m, m_wall,
                                          _dev(self.columns, torch.int32), _dev(self.normals), 1.7,
                                          periodic=(False, True), check=True)
        self.op = bo.channel_operator(ns, m, m_wall)
        n_b = self.columns.shape[0] // 2
        kind = np.array([bo.INFLOW] * n_b + [right] * n_b, dtype=np.int32)
        target = np.zeros((2 * n_b, 2))
        target[:n_b, 0] = u_in
        target[n_b:, 0] = C * C
        self.bnd = {"nodes": self.columns[:, 0], "normal": self.normals, "kind": kind, "target": target,
                    "L": ns.Lx, "mach": mach, "rho0": 1.0, "sigma": _sigma()}

    def plan(self, lb, dtype, oracle_weights=True):
        if oracle_weights:
            rp, col, w, kappa = self.op
            p = lb.Plan(_dev(rp, torch.int32), _dev(col, torch.int32), _dev(w), _dev(kappa), self.s, dtype=dtype)
        else:
            g = self.gop
            p = lb.Plan(g["row_ptr"], g["col"], g["w"], g["kappa"], self.s, dtype=dtype)
        b = self.bnd
        p.set_boundaries(_dev(b["nodes"], torch.int32), _dev(b["normal"]), _dev(b["kind"], torch.int32),
                         _dev(b["target"]), sigma=b["sigma"], L=b["L"], mach=b["mach"], rho0=b["rho0"])
        return p


@pytest.fixture(scope="module")
def box(lb):
    return Box(lb, 40, 12)


def _state(ns, seed=0, amp=0.02):
    q = np.zeros((3, ns.N))
    q[0] = amp * li.smooth_perturbation(ns.xy, kmax=3, seed=seed, Lx=ns.Lx, Ly=ns.Ly)
    q[1] = U0 + amp * C * li.smooth_perturbation(ns.xy, kmax=3, seed=seed + 1, Lx=ns.Lx, Ly=ns.Ly)
    q[2] = amp * C * li.smooth_perturbation(ns.xy, kmax=3, seed=seed + 2, Lx=ns.Lx, Ly=ns.Ly)
    return q


def test_open_box_operator_matches_oracle(box):
    ns = box.ns
    rp, col, w, kappa = box.op
    assert np.array_equal(box.gop["row_ptr"].cpu().numpy(), rp)
    assert np.array_equal(box.gop["col"].cpu().numpy(), col)
    assert box.gop["n_failed"] == 0
    wg = box.gop["w"].cpu().numpy()
    kg = box.gop["kappa"].cpu().numpy()
    row = ns.meta["row"]
    per = (False, True)
    rpc, colc = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=per)
    cond = {mm: oracle.build_weights(ns.xy, ns.h, ns.s, rpc, colc, mm, ns.Lx, ns.Ly, periodic=per,
                                     want_cond=True)["cond1"] for mm in (6, 4)}
    for i in range(ns.N):
        sl = slice(rp[i], rp[i + 1])
        a, b = wg[:, sl], w[:, sl]
        if row[i] >= 3:
            tol = max(50 * oracle.n_unknowns(6) * EPS64 * cond[6][i], 1e-13)
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), i
            continue
        assert np.abs(a[:2] - b[:2]).max() <= 1e-12 * np.abs(b[:2]).max(), i
        if row[i] == 0:
            assert np.abs(a[2:5] - b[2:5]).max() <= 1e-12 * np.abs(b[2:5]).max(), i
            assert np.all(a[5] == 0.0) and kg[i] == 0.0
        else:
            tol = max(50 * oracle.n_unknowns(4) * EPS64 * cond[4][i], 1e-13)
            assert np.abs(a[2:] - b[2:]).max() <= tol * np.abs(b[2:]).max(), i


def test_boundary_second_derivatives_exact_on_quartics(box):
    # the boundary nodes' second derivatives in the GPU-built operator (one-sided
    # five-point difference along the column, 1D LABFM of order 4 along the row, and
    # the column difference of the rows' tangential derivative for the mixed one) are
    # exact on every polynomial of total degree <= 4, on both boundaries
    ns = box.ns
    rp = box.gop["row_ptr"].cpu().numpy()
    col = box.gop["col"].cpu().numpy()
    w = box.gop["w"].cpu().numpy()
    rng = np.random.default_rng(3)
    ex = [(a, k - a) for k in range(5) for a in range(k + 1)]
    for _ in range(3):
        c = rng.standard_normal(len(ex))
        for i in box.bnd["nodes"]:
            sl = slice(rp[i], rp[i + 1])
            dx = ns.xy[col[sl], 0] - ns.xy[i, 0]
            dy = oracle.minimum_image(ns.xy[col[sl], 1] - ns.xy[i, 1], ns.Ly, True)
            p = sum(ck * dx ** a * dy ** b for ck, (a, b) in zip(c, ex))
            exact = (2 * c[ex.index((2, 0))], c[ex.index((1, 1))], 2 * c[ex.index((0, 2))])
            dp = p - c[0]  # difference form: p_j - p_i, p_i = p(0, 0)
            got = w[2:5, sl] @ dp
            scale = np.abs(w[2:5, sl]) @ np.abs(dp) + 1.0
            assert np.all(np.abs(got - exact) <= 1e-10 * scale), (i, got, exact)


def test_open_box_rhs_matches_oracle(lb, box):
    plan = box.plan(lb, torch.float64)
    q = _state(box.ns)
    R = lb.rhs(plan, _dev(q), lb.Phys(C * C, MU)).cpu().numpy()
    Ro = bo.boundary_rhs(q, box.op, box.bnd, C, MU)
    assert np.all(_rel_l2(R, Ro) <= 1e-12), _rel_l2(R, Ro)
    nb = box.bnd["nodes"]
    err = np.abs(R[:, nb] - Ro[:, nb]).max(axis=1) / np.abs(Ro[:, nb]).max(axis=1)
    assert np.all(err <= 1e-11), err
    plan.close()


def test_uniform_flow_is_steady_on_the_gpu(lb, box):
    plan = box.plan(lb, torch.float64)
    q = np.zeros((3, box.ns.N))
    q[1] = U0
    R = lb.rhs(plan, _dev(q), lb.Phys(C * C, MU)).cpu().numpy()
    assert np.all(R == 0.0)
    Q = _dev(q)
    lb.rk_step(plan, Q, 1e-3, 5, lb.Phys(C * C, MU))
    assert np.array_equal(Q.cpu().numpy(), q)
    plan.close()


def test_relaxation_rates_on_the_gpu(lb, box):
    # the closed forms of the oracle's pins: a uniform density excess relaxes at the
    # outflow by L4 = sigma/(2L) c (1 - M^2)(p - p_inf); a uniform velocity error at
    # the inflow by L4 = sigma rho0 c^2 (1 - M^2)/L du and L3 = sigma c/L dv
    plan = box.plan(lb, torch.float64)
    ns, b = box.ns, box.bnd
    sigma, M, L = b["sigma"], b["mach"], b["L"]
    out = b["nodes"][b["kind"] == bo.OUTFLOW]
    inn = b["nodes"][b["kind"] == bo.INFLOW]
    rho = 1.01
    q = np.zeros((3, ns.N))
    q[0], q[1] = np.log(rho), U0
    R = lb.rhs(plan, _dev(q), lb.Phys(C * C, MU)).cpu().numpy()
    L4 = sigma / (2 * L) * C * (1 - M * M) * (C * C * rho - C * C)
    assert np.allclose(R[0, out], -L4 / (rho * C * C), rtol=1e-12, atol=0)
    assert np.allclose(R[1, out], L4 / (rho * C), rtol=1e-12, atol=0)
    du, dv = 0.01, -0.02
    q = np.zeros((3, ns.N))
    q[1], q[2] = U0 + du, dv
    R = lb.rhs(plan, _dev(q), lb.Phys(C * C, MU)).cpu().numpy()
    L4 = sigma * C * C * (1 - M * M) / L * du
    L3 = sigma * C / L * dv
    assert np.allclose(R[0, inn], -L4 / (C * C), rtol=1e-12, atol=0)
    assert np.allclose(R[1, inn], -L4 / C, rtol=1e-12, atol=0)
    assert np.allclose(R[2, inn], -L3, rtol=1e-12, atol=0)
    plan.close()


def test_open_box_time_steps_match_oracle(lb, box):
    # ten steps (interior eq. icns, boundary rows, LODI inflow and outflow, filter
    # off the boundary nodes): the change over the steps within 1e-12
    ns = box.ns
    plan = box.plan(lb, torch.float64)
    q0 = _state(ns, seed=5)
    dt = 0.5 * oracle.stable_dt(q0, ns.s, C, MU)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 10, lb.Phys(C * C, MU))
    qo = q0
    for _ in range(10):
        qo = bo.boundary_time_step(qo, dt, box.op, box.bnd, C, MU)
    qg = Q.cpu().numpy()
    assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-12), _rel_l2(qg - q0, qo - q0)
    plan.close()


def test_open_box_gpu_operator_and_fp32(lb, box):
    # the GPU-built operator (weights within the weight build's conditioning bound of
    # the oracle's, test above) stepped on the GPU against the oracle's step with those
    # same weights: FP64 to 1e-12 over three steps, FP32 one step within
    # the derived step budget
    from tests.fp32_budget import boundary_step_bound
    ns = box.ns
    q0 = _state(ns, seed=8)
    dt = 0.5 * oracle.stable_dt(q0, ns.s, C, MU)
    gop = (box.gop["row_ptr"].cpu().numpy(), box.gop["col"].cpu().numpy(), box.gop["w"].cpu().numpy(),
           box.gop["kappa"].cpu().numpy())
    q1 = bo.boundary_time_step(q0, dt, gop, box.bnd, C, MU)
    qo = q0
    for _ in range(3):
        qo = bo.boundary_time_step(qo, dt, gop, box.bnd, C, MU)
    plan = box.plan(lb, torch.float64, oracle_weights=False)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 3, lb.Phys(C * C, MU))
    plan.close()
    qg = Q.cpu().numpy()
    assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-12), _rel_l2(qg - q0, qo - q0)
    plan = box.plan(lb, torch.float32, oracle_weights=False)
    Q = _dev(q0, torch.float32)
    lb.rk_step(plan, Q, dt, 1, lb.Phys(C * C, MU))
    plan.close()
    B = boundary_step_bound(q0, q1, dt, gop[2], gop[3], gop[0], gop[1], box.bnd, C, MU)
    ratio = np.abs(Q.double().cpu().numpy() - q1) / np.where(B > 0, B, np.inf)
    print("FP32 open-box step, GPU operator: max error / budget", ratio.max())
    assert ratio.max() <= 1.0, ratio.max()


def _pulse(lb, right, nx=96, ny=12):
    # a right-going acoustic pulse (u' = c a') in fluid at rest, inflow at zero
    # velocity on the left; run until a reflected pulse would be a quarter of the
    # box back from the right boundary
    bx = Box(lb, nx, ny, seed=2, right=right, u_in=0.0, mach=0.0)
    ns = bx.ns
    plan = bx.plan(lb, torch.float64, oracle_weights=False)
    A, x0, w = 1e-3, 0.6 * ns.Lx, 0.3
    x = ns.xy[:, 0]
    pulse = A * np.exp(-((x - x0) / w) ** 2)
    q = np.zeros((3, ns.N))
    q[0] = pulse
    q[1] = C * pulse
    dt = oracle.stable_dt(q, ns.s, C, MU)
    n = int(np.ceil((ns.Lx - x0 + 0.25 * ns.Lx) / C / dt))
    Q = _dev(q)
    lb.rk_step(plan, Q, dt, n, lb.Phys(C * C, MU))
    qg = Q.cpu().numpy()
    plan.close()
    away = (x > 0.2 * ns.Lx) & (x < 0.85 * ns.Lx)
    return float(np.abs(qg[0][away]).max()) / A, qg


def test_acoustic_pulse_leaves_through_the_outflow_on_the_gpu(lb):
    out, q = _pulse(lb, bo.OUTFLOW)
    wall, _ = _pulse(lb, bo.WALL)
    print("pulse left behind (outflow, wall):", out, wall)
    assert np.all(np.isfinite(q))
    assert 0.8 < wall < 1.2, wall
    assert out < 0.05, out


def test_boundary_arguments_are_checked(lb, box):
    plan = box.plan(lb, torch.float64)
    b = box.bnd
    nodes, normal = _dev(b["nodes"], torch.int32), _dev(b["normal"])
    kind, target = _dev(b["kind"], torch.int32), _dev(b["target"])
    bad = b["kind"].copy()
    bad[0] = 7
    with pytest.raises(lb.LabfmError):
        plan.set_boundaries(nodes, normal, _dev(bad, torch.int32), target)
    for kw in ({"sigma": -1.0}, {"L": 0.0}, {"mach": 1.0}, {"rho0": 0.0}):
        with pytest.raises(lb.LabfmError):
            plan.set_boundaries(nodes, normal, kind, target, **kw)
    # the refused calls leave no boundaries: eq. icns everywhere
    q = _state(box.ns)
    R = lb.rhs(plan, _dev(q), lb.Phys(C * C, MU)).cpu().numpy()
    rp, col, w, _ = box.op
    assert np.all(_rel_l2(R, oracle.rhs(q, w[:5], rp, col, C * C, MU)) <= 1e-12)
    plan.close()


def test_lamb_oseen_workload_sampled(lb):
    # the finest box of the Lamb-Oseen study (R_c/s = 16: 400 x 400, 160,400 nodes):
    # the GPU-built operator at sampled rows of every kind against the oracle's rows,
    # and the FP64 right-hand side of the vortex state (inflow and outflow active) at
    # those rows against the oracle with the same weights, to 1e-12
    from tests import lamb_oseen as lo
    n = 400
    ns = li.open_box(n, n, m=6, jitter=0.05, seed=0)
    cols, normals = li.channel_walls(ns)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    gop = lb.build_wall_operator(xy, h, s, ns.Lx, ns.Ly, 6, 4, _dev(cols, torch.int32), _dev(normals), 1.7,
                                 periodic=(False, True), check=True)
    assert gop["n_failed"] == 0
    rng = np.random.default_rng(31)
    row = ns.meta["row"]
    pick = [rng.choice(np.flatnonzero(row == q), 8, replace=False) for q in range(5)]
    pick.append(rng.choice(np.flatnonzero(row == 5), 16, replace=False))
    rows = np.unique(np.concatenate(pick))
    rp_o, col_o, w_o, _ = bo.channel_operator(ns, 6, 4, rows=rows)
    rp = gop["row_ptr"].cpu().numpy()
    col = gop["col"].cpu().numpy()
    w = gop["w"].cpu().numpy()
    for k, i in enumerate(rows):
        sl, so = slice(rp[i], rp[i + 1]), slice(rp_o[k], rp_o[k + 1])
        assert np.array_equal(col[sl], col_o[so]), i
        if row[i] <= 2:
            assert np.abs(w[:2, sl] - w_o[:2, so]).max() <= 1e-12 * np.abs(w_o[:2, so]).max(), i
    c = 1.0 / li.LAMB_OSEEN_MACH
    mu = li.LAMB_OSEEN_RC_OVER_H / li.LAMB_OSEEN_RE
    q = li.lamb_oseen_fields(ns.xy, c, centre=(0.5 * ns.Lx, 0.5))
    n_b = cols.shape[0] // 2
    kind = np.array([bo.INFLOW] * n_b + [bo.OUTFLOW] * n_b, dtype=np.int32)
    target = np.zeros((2 * n_b, 2))
    target[:n_b, 0] = 1.0
    target[n_b:, 0] = c * c
    bnd = {"nodes": cols[:, 0], "normal": normals, "kind": kind, "target": target, "L": ns.Lx,
           "mach": li.LAMB_OSEEN_MACH, "rho0": 1.0, "sigma": lo.sigma()}
    plan = lb.Plan(gop["row_ptr"], gop["col"], gop["w"], gop["kappa"], s, dtype=torch.float64)
    plan.set_boundaries(_dev(bnd["nodes"], torch.int32), _dev(normals), _dev(kind, torch.int32), _dev(target),
                        sigma=bnd["sigma"], L=bnd["L"], mach=bnd["mach"], rho0=1.0)
    # perturb the far field so that the boundary terms are not at rest
    q[1] += 0.01 * li.smooth_perturbation(ns.xy, kmax=3, seed=2, Lx=ns.Lx, Ly=ns.Ly)
    R = lb.rhs(plan, _dev(q), lb.Phys(c * c, mu)).cpu().numpy()
    plan.close()
    cnt = np.zeros(ns.N, dtype=np.int64)
    cnt[rows] = rp[rows + 1] - rp[rows]
    rps = np.concatenate([[0], np.cumsum(cnt)])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    Ro = bo.boundary_rhs(q, (rps, col[idx], w[:, idx], None), bnd, c, mu)
    for f in range(3):
        err = np.abs(R[f][rows] - Ro[f][rows]).max() / np.abs(Ro[f][rows]).max()
        assert err <= 1e-12, (f, err)


def test_open_box_fp32_rhs_within_derived_budget(lb, box):
    # one FP32 right-hand side (FP32 state, nondimensional FP32 weights) against the
    # FP64 oracle with the same operator, elementwise within the budget derived in
    # tests/fp32_budget.py (eq. icns off the boundary, the linearised inflow and
    # outflow formulas on it)
    from tests.fp32_budget import boundary_rhs_bound
    plan = box.plan(lb, torch.float32)
    q = _state(box.ns, seed=11)
    R = lb.rhs(plan, _dev(q, torch.float32), lb.Phys(C * C, MU)).double().cpu().numpy()
    plan.close()
    Ro = bo.boundary_rhs(q, box.op, box.bnd, C, MU)
    rp, col, w, _ = box.op
    B = boundary_rhs_bound(q, w, rp, col, box.bnd, C, MU)
    ratio = np.abs(R - Ro) / B
    nb = box.bnd["nodes"]
    print("FP32 open box: max error / budget, all nodes", ratio.max(), "boundary nodes", ratio[:, nb].max())
    assert ratio.max() <= 1.0, ratio.max()


def test_open_box_fp32_step_within_derived_budget(lb, box):
    # one FP32 time step (oracle operator) against the FP64 oracle step, elementwise
    # within the step budget derived from the right-hand-side budget
    from tests.fp32_budget import boundary_step_bound
    ns = box.ns
    q0 = _state(ns, seed=13)
    dt = 0.5 * oracle.stable_dt(q0, ns.s, C, MU)
    q1 = bo.boundary_time_step(q0, dt, box.op, box.bnd, C, MU)
    plan = box.plan(lb, torch.float32)
    Q = _dev(q0, torch.float32)
    lb.rk_step(plan, Q, dt, 1, lb.Phys(C * C, MU))
    plan.close()
    rp, col, w, kappa = box.op
    B = boundary_step_bound(q0, q1, dt, w, kappa, rp, col, box.bnd, C, MU)
    ratio = np.abs(Q.double().cpu().numpy() - q1) / B
    print("FP32 open-box step: max error / budget", ratio.max())
    assert ratio.max() <= 1.0, ratio.max()
