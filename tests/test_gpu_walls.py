"""The boundary row on the GPU (Section 7.1, Appendix A) against the oracle's
channel: the wall operator (LABFM inside, five-point differences and 1D LABFM on
the wall rows, rotated), the no-slip wall's right-hand side in LODI form, whole
time steps, and the Poiseuille start-up of Section 8.2 converging to the analytic
solution at the oracle's order."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import boundary_oracle as bo
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


def _rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


class Channel:
    """A channel node set with the oracle's operator and the GPU-built one."""

    def __init__(self, lb, nx, ny, m=6, m_wall=4, jitter=0.1, seed=0):
        self.ns = ns = li.channel(nx, ny, m=m, jitter=jitter, seed=seed)
        self.m, self.m_wall = m, m_wall
        self.columns, self.normals = li.channel_walls(ns)
        self.xy, self.h, self.s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
        self.gop = lb.build_wall_operator(self.xy, self.h, self.s, ns.Lx, ns.Ly, m, m_wall,
                                          _dev(self.columns, torch.int32), _dev(self.normals), 1.7,
                                          periodic=(True, False), check=True)
        self.op = bo.channel_operator(ns, m, m_wall)
        self.wall_nodes = self.columns[:, 0]

    def plan(self, lb, dtype, oracle_weights=True):
        if oracle_weights:
            rp, col, w, kappa = self.op
            p = lb.Plan(_dev(rp, torch.int32), _dev(col, torch.int32), _dev(w), _dev(kappa), self.s, dtype=dtype)
        else:
            g = self.gop
            p = lb.Plan(g["row_ptr"], g["col"], g["w"], g["kappa"], self.s, dtype=dtype)
        p.set_walls(_dev(self.wall_nodes, torch.int32), _dev(self.normals))
        return p


@pytest.fixture(scope="module")
def ch(lb):
    return Channel(lb, 20, 18, seed=3)


def test_wall_operator_stencils_bit_exact(ch):
    rp, col, _, _ = ch.op
    assert np.array_equal(ch.gop["row_ptr"].cpu().numpy(), rp)
    assert np.array_equal(ch.gop["col"].cpu().numpy(), col)
    assert ch.gop["n_failed"] == 0


def test_wall_operator_weights_match_oracle(ch):
    # LABFM rows within the conditioning bound of the weight build (the LU is
    # backward stable; the two sides differ in summation order), strip first
    # derivatives (five-point differences and a 4 x 4 1D LABFM system) to 1e-12
    ns = ch.ns
    rp, col, w, kappa = ch.op
    wg = ch.gop["w"].cpu().numpy()
    kg = ch.gop["kappa"].cpu().numpy()
    row = ns.meta["row"]
    rpc, colc = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=(True, False))
    cond = {}
    for mm in {ch.m, ch.m_wall}:
        cond[mm] = oracle.build_weights(ns.xy, ns.h, ns.s, rpc, colc, mm, ns.Lx, ns.Ly, periodic=(True, False),
                                        want_cond=True)["cond1"]
    n = {mm: oracle.n_unknowns(mm) for mm in cond}
    for i in range(ns.N):
        sl = slice(rp[i], rp[i + 1])
        a, b = wg[:, sl], w[:, sl]
        if row[i] >= 3:
            tol = max(50 * n[ch.m] * EPS64 * cond[ch.m][i], 1e-13)
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), i
            assert abs(kg[i] - kappa[i]) <= tol * abs(kappa[i]), i
            continue
        # strip first derivatives
        assert np.abs(a[:2] - b[:2]).max() <= 1e-12 * np.abs(b[:2]).max(), i
        if row[i] == 0:
            # "FD + 1D-LABFM" second derivatives; the boundary node is not filtered
            assert np.abs(a[2:5] - b[2:5]).max() <= 1e-12 * np.abs(b[2:5]).max(), i
            assert np.all(a[5] == 0.0) and kg[i] == 0.0
        else:
            tol = max(50 * n[ch.m_wall] * EPS64 * cond[ch.m_wall][i], 1e-13)
            assert np.abs(a[2:] - b[2:]).max() <= tol * np.abs(b[2:]).max(), i
            assert abs(kg[i] - kappa[i]) <= tol * abs(kappa[i]), i


def test_wall_rows_differentiate_quartics_exactly(ch):
    # Section 7.1: the wall rows' first derivatives are exact on every polynomial of
    # total degree <= 4 (five-point differences, 4th-order 1D LABFM), in the GPU's
    # operator on both walls
    ns = ch.ns
    rp = ch.gop["row_ptr"].cpu().numpy()
    col = ch.gop["col"].cpu().numpy()
    w = ch.gop["w"].cpu().numpy()
    strip = np.flatnonzero(ns.meta["row"] <= 2)
    rng = np.random.default_rng(7)
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    for _ in range(4):
        c = rng.standard_normal(15)
        ex = [(a, k - a) for k in range(5) for a in range(k + 1)]
        # a local polynomial around each node (the channel is periodic in x: no wrap
        # within the uniform rows' supports except across x = 0, handled by offsets)
        for i in strip:
            sl = slice(rp[i], rp[i + 1])
            dx = oracle.minimum_image(x[col[sl]] - x[i], ns.Lx, True)
            dy = y[col[sl]] - y[i]
            p = sum(ck * dx ** a * dy ** b for ck, (a, b) in zip(c, ex))
            px = c[ex.index((1, 0))]
            py = c[ex.index((0, 1))]
            dp = p - c[0]  # difference form: p_j - p_i, p_i = p(0, 0)
            scale = (np.abs(w[0, sl]).sum() + np.abs(w[1, sl]).sum()) * np.abs(dp).max() + 1.0
            assert abs(np.dot(w[0, sl], dp) - px) <= 1e-11 * scale, i
            assert abs(np.dot(w[1, sl], dp) - py) <= 1e-11 * scale, i


@pytest.mark.parametrize("g", [(0.0, 0.0), (0.3, -0.2)])
def test_channel_rhs_matches_oracle(lb, ch, g):
    ns = ch.ns
    plan = ch.plan(lb, torch.float64)
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=4)
    q[1:, ch.wall_nodes] = 0.0  # no slip
    R = lb.rhs(plan, _dev(q), lb.Phys(100.0, 0.01, g[0], g[1])).cpu().numpy()
    Ro = bo.channel_rhs(q, ch.op, ns, 10.0, 0.01, g)
    assert np.all(_rel_l2(R, Ro) <= 1e-12), _rel_l2(R, Ro)
    assert np.all(R[1:, ch.wall_nodes] == 0.0)
    plan.close()


def test_channel_time_steps_match_oracle(lb, ch):
    # ten steps of the channel (interior eq. icns, wall rows, LODI wall, filter off
    # the wall) from a perturbed state: the change over the steps within 1e-12
    ns = ch.ns
    c, mu, g = 10.0, 0.01, (0.5, 0.0)
    plan = ch.plan(lb, torch.float64)
    q0 = np.zeros((3, ns.N))
    q0[0] = 0.02 * li.smooth_perturbation(ns.xy, kmax=3, seed=9, Ly=ns.Ly)
    q0[1] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=10, Ly=ns.Ly)
    q0[1:, ch.wall_nodes] = 0.0
    dt = 0.5 * oracle.stable_dt(np.stack([q0[0], q0[1] + 1.0, q0[2]]), ns.s, c, mu)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 10, lb.Phys(c * c, mu, g[0], g[1]))
    qo = q0
    for _ in range(10):
        qo = bo.channel_time_step(qo, dt, ch.op, ns, c, mu, g)
    qg = Q.cpu().numpy()
    assert np.all(qg[1:, ch.wall_nodes] == 0.0)
    assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-12), _rel_l2(qg - q0, qo - q0)
    plan.close()


def test_channel_step_with_gpu_operator_and_fp32(lb, ch):
    # the GPU-built operator (whose weights match the oracle's within the weight
    # build's conditioning bound, test above) stepped on the GPU against the oracle's
    # step with those same weights: FP64 to 1e-12, FP32 one step within
    # the derived step budget; the wall velocity stays exactly zero
    from tests.fp32_budget import boundary_step_bound
    ns = ch.ns
    c, mu, g = 10.0, 0.01, (0.5, 0.0)
    q0 = np.zeros((3, ns.N))
    q0[0] = 0.02 * li.smooth_perturbation(ns.xy, kmax=3, seed=9, Ly=ns.Ly)
    q0[1] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=10, Ly=ns.Ly)
    q0[1:, ch.wall_nodes] = 0.0
    dt = 0.5 * oracle.stable_dt(np.stack([q0[0], q0[1] + 1.0, q0[2]]), ns.s, c, mu)
    gop = (ch.gop["row_ptr"].cpu().numpy(), ch.gop["col"].cpu().numpy(), ch.gop["w"].cpu().numpy(),
           ch.gop["kappa"].cpu().numpy())
    q1 = bo.channel_time_step(q0, dt, gop, ns, c, mu, g)
    qo = q0
    for _ in range(3):
        qo = bo.channel_time_step(qo, dt, gop, ns, c, mu, g)
    phys = lb.Phys(c * c, mu, g[0], g[1])
    plan = ch.plan(lb, torch.float64, oracle_weights=False)
    Q = _dev(q0)
    lb.rk_step(plan, Q, dt, 3, phys)
    plan.close()
    qg = Q.cpu().numpy()
    assert np.all(qg[1:, ch.wall_nodes] == 0.0)
    assert np.all(_rel_l2(qg - q0, qo - q0) <= 1e-12), _rel_l2(qg - q0, qo - q0)
    plan = ch.plan(lb, torch.float32, oracle_weights=False)
    Q = _dev(q0, torch.float32)
    lb.rk_step(plan, Q, dt, 1, phys)
    plan.close()
    got = Q.double().cpu().numpy()
    assert np.all(got[1:, ch.wall_nodes] == 0.0)
    bnd = {"nodes": ch.wall_nodes, "normal": ch.normals, "kind": np.zeros(len(ch.wall_nodes), dtype=np.int32),
           "target": np.zeros((len(ch.wall_nodes), 2)), "L": 1.0, "mach": 0.0, "rho0": 1.0}
    B = boundary_step_bound(q0, q1, dt, gop[2], gop[3], gop[0], gop[1], bnd, c, mu, g)
    ratio = np.abs(got - q1) / np.where(B > 0, B, np.inf)
    print("FP32 channel step, GPU operator: max error / budget", ratio.max())
    assert ratio.max() <= 1.0, ratio.max()


def _poiseuille_start_up(y, t, H, g, nu, nterms=400):
    u = g / (2 * nu) * y * (H - y)
    for k in range(nterms):
        n = 2 * k + 1
        u = u - (4 * g * H * H / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y / H)
                 * np.exp(-(n * np.pi) ** 2 * nu * t / H ** 2))
    return u


def _poiseuille_error(lb, nx, dtype=torch.float64, jitter=0.1):
    # Section 8.2: Re = 10, Ma = 0.05, from rest, velocity error at t U0 / H = 1
    ch = Channel(lb, nx, nx, m=6, m_wall=4, jitter=jitter)
    ns = ch.ns
    H, U0 = ns.Ly, 1.0
    mu = U0 * H / 10.0
    g = 8 * mu * U0 / H ** 2
    c = U0 / 0.05
    plan = ch.plan(lb, dtype, oracle_weights=False)
    q = np.zeros((3, ns.N))
    dt0 = oracle.stable_dt(np.stack([q[0], q[1] + U0, q[2]]), ns.s, c, mu)
    nsteps = int(np.ceil(1.0 / dt0))
    Q = _dev(q, dtype)
    lb.rk_step(plan, Q, 1.0 / nsteps, nsteps, lb.Phys(c * c, mu, g, 0.0))
    qg = Q.double().cpu().numpy()
    plan.close()
    ua = _poiseuille_start_up(ns.xy[:, 1], 1.0, H, g, mu)
    assert np.all(qg[1:, ch.wall_nodes] == 0.0)
    return np.linalg.norm(qg[1] - ua) / np.linalg.norm(ua), float(np.abs(qg[2]).max())


def test_poiseuille_start_up_converges_on_the_gpu(lb):
    # the oracle's pin (order > 4 from s = H/16 to H/24, interior jitter +-0.1 s) on
    # the GPU path; finer channels at +-0.05 s jitter, where the sixth-order filter
    # stays stable over the ~1000 steps of s = H/48 (at +-0.1 s the filter of some
    # m = 6 stencils amplifies a mode: the run goes non-finite, as in the periodic case)
    errs = {nx: _poiseuille_error(lb, nx) for nx in (16, 24)}
    errs.update({(nx, 0.05): _poiseuille_error(lb, nx, jitter=0.05) for nx in (24, 48)})
    e = {k: v[0] for k, v in errs.items()}
    assert e[16] < 3e-3 and e[24] < 4e-4, e
    assert np.log(e[16] / e[24]) / np.log(24 / 16) > 4.0, e
    assert np.log(e[(24, 0.05)] / e[(48, 0.05)]) / np.log(2.0) > 3.5, e
    assert all(v[1] < 1e-3 for v in errs.values())
    # FP32: the same error as FP64 at this resolution (FP32 rounding is far below it)
    e32, _ = _poiseuille_error(lb, 24, torch.float32)
    print("Poiseuille start-up errors (FP64):", e, "FP32 at 24:", e32)
    assert abs(e32 / e[24] - 1.0) < 0.2, (e32, e[24])


def test_wall_arguments_are_checked(lb, ch):
    ns = ch.ns
    plan = ch.plan(lb, torch.float64)
    nodes = _dev(ch.wall_nodes, torch.int32)
    with pytest.raises(lb.LabfmError):  # a node listed twice
        plan.set_walls(torch.cat([nodes[:3], nodes[:1]]), _dev(ch.normals[:4]))
    bad = ch.normals.copy()
    bad[0] *= 1.1
    with pytest.raises(lb.LabfmError):  # not a unit normal
        plan.set_walls(nodes, _dev(bad))
    # the failed calls leave no walls; set them again, then the adjoint refuses
    plan.set_walls(nodes, _dev(ch.normals))
    lb.enable_adjoint(plan)
    with pytest.raises(lb.LabfmError):
        lb.rhs_adjoint(plan, _dev(np.zeros((3, ns.N))), _dev(np.zeros((3, ns.N))), lb.Phys(100.0, 0.01))
    # removing the walls restores eq. icns everywhere
    plan.set_walls(torch.empty(0, dtype=torch.int32, device="cuda"), torch.empty((0, 2), dtype=torch.float64,
                                                                                  device="cuda"))
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=4)
    R = lb.rhs(plan, _dev(q), lb.Phys(100.0, 0.01)).cpu().numpy()
    rp, col, w, _ = ch.op
    assert np.all(_rel_l2(R, oracle.rhs(q, w[:5], rp, col, 100.0, 0.01)) <= 1e-12)
    # columns: a node in two columns, and an out-of-range node
    cols = ch.columns.copy()
    cols[1, 2] = cols[0, 2]
    with pytest.raises(lb.LabfmError):
        lb.build_wall_operator(ch.xy, ch.h, ch.s, ns.Lx, ns.Ly, 6, 4, _dev(cols, torch.int32), _dev(ch.normals))
    cols = ch.columns.copy()
    cols[0, 4] = ns.N
    with pytest.raises(lb.LabfmError):
        lb.build_wall_operator(ch.xy, ch.h, ch.s, ns.Lx, ns.Ly, 6, 4, _dev(cols, torch.int32), _dev(ch.normals))
    plan.close()


# ---------------------------------------------------------------- the channel workload, sampled

@pytest.fixture(scope="module")
def ch512(lb):
    # the bench's channel: 512 x 512, +-0.05 s jitter inside, m = 6 inside, m = 4 on the
    # wall rows; the GPU-built operator; sampled rows of every kind
    ns = li.channel(512, 512, m=6, jitter=0.05)
    cols, normals = li.channel_walls(ns)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    gop = lb.build_wall_operator(xy, h, s, ns.Lx, ns.Ly, 6, 4, _dev(cols, torch.int32), _dev(normals), 1.7,
                                 periodic=(True, False), check=True)
    rng = np.random.default_rng(21)
    row = ns.meta["row"]
    pick = [rng.choice(np.flatnonzero(row == q), 12, replace=False) for q in range(5)]
    pick.append(rng.choice(np.flatnonzero(row == 5), 24, replace=False))
    rows = np.unique(np.concatenate(pick + [[0, ns.N - 1]]))
    return dict(ns=ns, cols=cols, normals=normals, s=s, gop=gop, rows=rows,
                op=bo.channel_operator(ns, 6, 4, rows=rows))


def test_channel_workload_operator_rows_sampled(ch512):
    ns, rows, gop = ch512["ns"], ch512["rows"], ch512["gop"]
    rp_o, col_o, w_o, k_o = ch512["op"]
    rp = gop["row_ptr"].cpu().numpy()
    col = gop["col"].cpu().numpy()
    w = gop["w"].cpu().numpy()
    kap = gop["kappa"].cpu().numpy()
    assert gop["n_failed"] == 0
    per = (True, False)
    rpn, coln = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=per, rows=rows)
    cond = {mm: oracle.build_weights(ns.xy, ns.h, ns.s, rpn, coln, mm, ns.Lx, ns.Ly, periodic=per, rows=rows,
                                     want_cond=True)["cond1"] for mm in (6, 4)}
    row = ns.meta["row"]
    for k, i in enumerate(rows):
        sl, so = slice(rp[i], rp[i + 1]), slice(rp_o[k], rp_o[k + 1])
        assert np.array_equal(col[sl], col_o[so]), i
        a, b = w[:, sl], w_o[:, so]
        if row[i] >= 3:
            tol = max(50 * oracle.n_unknowns(6) * EPS64 * cond[6][k], 1e-13)
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), i
            assert abs(kap[i] - k_o[k]) <= tol * abs(k_o[k]), i
            continue
        assert np.abs(a[:2] - b[:2]).max() <= 1e-12 * np.abs(b[:2]).max(), i
        if row[i] == 0:
            assert np.abs(a[2:5] - b[2:5]).max() <= 1e-12 * np.abs(b[2:5]).max(), i
            assert np.all(a[5] == 0.0) and kap[i] == 0.0
        else:
            tol = max(50 * oracle.n_unknowns(4) * EPS64 * cond[4][k], 1e-13)
            assert np.abs(a[2:] - b[2:]).max() <= tol * np.abs(b[2:]).max(), i


def test_channel_workload_rhs_sampled(lb, ch512):
    # FP64 right-hand side of the bench's channel at the sampled rows against the oracle
    # with the same (GPU-built) weights, to 1e-12; and the FP32 plan in the bench's launch
    # shape within the FP32 budget at the sampled rows that follow eq. icns
    from tests.fp32_budget import U32, rhs_bound
    ns, rows, gop = ch512["ns"], ch512["rows"], ch512["gop"]
    c, mu, g = 20.0, 0.1, (0.5, 0.0)
    q = np.zeros((3, ns.N))
    q[0] = 0.01 * li.smooth_perturbation(ns.xy, kmax=4, seed=3, Ly=ns.Ly)
    q[1] = 0.5 * li.smooth_perturbation(ns.xy, kmax=4, seed=4, Ly=ns.Ly)
    q[2] = 0.1 * li.smooth_perturbation(ns.xy, kmax=4, seed=5, Ly=ns.Ly)
    wall = ch512["cols"][:, 0]
    q[1:, wall] = 0.0
    rp = gop["row_ptr"].cpu().numpy()
    col = gop["col"].cpu().numpy()
    w = gop["w"].cpu().numpy()
    cnt = np.zeros(ns.N, dtype=np.int64)
    cnt[rows] = rp[rows + 1] - rp[rows]
    rps = np.concatenate([[0], np.cumsum(cnt)])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    bnd = {"nodes": wall, "normal": ch512["normals"], "kind": np.zeros(len(wall), dtype=np.int32),
           "target": np.zeros((len(wall), 2)), "L": 1.0, "mach": 0.0, "rho0": 1.0}
    Ro = bo.boundary_rhs(q, (rps, col[idx], w[:, idx], None), bnd, c, mu, g)
    phys = lb.Phys(c * c, mu, g[0], g[1])
    for dtype in (torch.float64, torch.float32):
        plan = lb.Plan(gop["row_ptr"], gop["col"], gop["w"], gop["kappa"], ch512["s"], dtype=dtype)
        plan.set_walls(_dev(wall, torch.int32), _dev(ch512["normals"]))
        plan.set_launch(4, 128)  # the channel bench's tuned shape (walls run the plain grid)
        R = lb.rhs(plan, _dev(q, dtype), phys).double().cpu().numpy()
        plan.close()
        if dtype == torch.float64:
            for f in range(3):
                err = np.abs(R[f][rows] - Ro[f][rows]).max() / np.abs(Ro[f][rows]).max()
                assert err <= 1e-12, (f, err)
            assert np.all(R[1:, wall] == 0.0)
        else:
            icns = rows[ns.meta["row"][rows] > 0]
            B = rhs_bound(q, w[:, idx], rps, col[idx], c * c, mu)
            # the body force enters each momentum sum once more: its rounding and that
            # of the final addition
            B[1] += 4 * U32 * abs(g[0])
            B[2] += 4 * U32 * abs(g[1])
            ratio = np.abs(R[:, icns] - Ro[:, icns]) / B[:, icns]
            assert ratio.max() <= 1.0, ratio.max()


@pytest.mark.parametrize("g", [(0.0, 0.0), (0.3, -0.2)])
def test_channel_fp32_rhs_within_derived_budget(lb, ch, g):
    # one FP32 right-hand side of the channel (no-slip walls in LODI form) against
    # the FP64 oracle with the same operator, elementwise within the budget derived in
    # tests/fp32_budget.py
    from tests.fp32_budget import boundary_rhs_bound
    ns = ch.ns
    plan = ch.plan(lb, torch.float32)
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=4)
    q[1:, ch.wall_nodes] = 0.0
    R = lb.rhs(plan, _dev(q, torch.float32), lb.Phys(100.0, 0.01, g[0], g[1])).double().cpu().numpy()
    plan.close()
    Ro = bo.channel_rhs(q, ch.op, ns, 10.0, 0.01, g)
    rp, col, w, _ = ch.op
    bnd = {"nodes": ch.wall_nodes, "normal": ch.normals, "kind": np.zeros(len(ch.wall_nodes), dtype=np.int32),
           "target": np.zeros((len(ch.wall_nodes), 2)), "L": 1.0, "mach": 0.0, "rho0": 1.0}
    B = boundary_rhs_bound(q, w, rp, col, bnd, 10.0, 0.01, g)
    ratio = np.abs(R - Ro) / np.where(B > 0, B, np.inf)
    assert np.all(R[1:, ch.wall_nodes] == 0.0)
    print("FP32 channel: max error / budget", ratio.max(), "walls", ratio[0, ch.wall_nodes].max())
    assert ratio.max() <= 1.0, ratio.max()


def test_channel_fp32_step_within_derived_budget(lb, ch):
    # one FP32 time step of the channel (oracle operator, gravity on) against the FP64
    # oracle step within the derived step budget; the wall velocity stays exactly zero
    from tests.fp32_budget import boundary_step_bound
    ns = ch.ns
    c, mu, g = 10.0, 0.01, (0.5, 0.0)
    q0 = np.zeros((3, ns.N))
    q0[0] = 0.02 * li.smooth_perturbation(ns.xy, kmax=3, seed=9, Ly=ns.Ly)
    q0[1] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=10, Ly=ns.Ly)
    q0[1:, ch.wall_nodes] = 0.0
    dt = 0.5 * oracle.stable_dt(np.stack([q0[0], q0[1] + 1.0, q0[2]]), ns.s, c, mu)
    q1 = bo.channel_time_step(q0, dt, ch.op, ns, c, mu, g)
    plan = ch.plan(lb, torch.float32)
    Q = _dev(q0, torch.float32)
    lb.rk_step(plan, Q, dt, 1, lb.Phys(c * c, mu, g[0], g[1]))
    plan.close()
    rp, col, w, kappa = ch.op
    bnd = {"nodes": ch.wall_nodes, "normal": ch.normals, "kind": np.zeros(len(ch.wall_nodes), dtype=np.int32),
           "target": np.zeros((len(ch.wall_nodes), 2)), "L": 1.0, "mach": 0.0, "rho0": 1.0}
    B = boundary_step_bound(q0, q1, dt, w, kappa, rp, col, bnd, c, mu, g)
    got = Q.double().cpu().numpy()
    assert np.all(got[1:, ch.wall_nodes] == 0.0)
    ratio = np.abs(got - q1) / np.where(B > 0, B, np.inf)
    print("FP32 channel step: max error / budget", ratio.max())
    assert ratio.max() <= 1.0, ratio.max()
