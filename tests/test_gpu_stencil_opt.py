"""Stencil optimisation (Section 4) and the modal response of built operators
(Section 3) on the GPU against the FP64 oracle."""
import math

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_modal_response_matches_oracle(lb):
    # ragged: 37 x 29 nodes with +-0.3 s jitter, sixth order, oracle weights on both sides
    ns = li.tgv_lattice(37, 29, m=6, h_over_s=2.2, jitter=0.3, seed=61)
    rp, col = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    w = oracle.build_weights(ns.xy, ns.h, ns.s, rp, col, 6, ns.Lx, ns.Ly)["w"]
    ref = oracle.modal_response(ns.xy, ns.s, rp, col, w, ns.Lx, ns.Ly, nk=16)
    got = lb.modal_response(_dev(ns.xy), _dev(ns.s), ns.Lx, ns.Ly, _dev(rp, torch.int32),
                            _dev(col, torch.int32), _dev(w), nk=16).cpu().numpy()
    # |A| ~ 1 built from sums of |w| |sin| ~ n_j |w| s: rounding ~1e-14 of that
    assert np.max(np.abs(got - ref)) <= 1e-10, np.max(np.abs(got - ref))


def test_modal_response_full_size_sampled(lb):
    # 512 x 512, m = 8, GPU-built weights; sampled rows against the oracle's
    # per-node response on the same weights, and the low-wavenumber limit at every node
    ns = li.tgv_lattice(512, m=8, jitter=0.1, seed=62)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 8, check=True)
    A = lb.modal_response(xy, s, ns.Lx, ns.Ly, rp, col, wb["w"], nk=64)
    # eighth-order operators: response 1 to ~(k s)^8 at k = k_Ny / 64
    assert float((A[:, :, 0] - 1.0).abs().max()) < 1e-7
    rows = np.random.default_rng(5).choice(ns.N, 40, replace=False)
    rpn, coln, w = rp.cpu().numpy(), col.cpu().numpy(), wb["w"].cpu().numpy()
    An = A.cpu().numpy()
    for i in rows:
        sl = slice(rpn[i], rpn[i + 1])
        dx, dy = oracle.offsets(ns.xy, np.full(rpn[i + 1] - rpn[i], i), coln[sl], ns.Lx, ns.Ly)
        ref = oracle.amplitude_response(dx, dy, ns.s[i], w[0][sl], w[1][sl], w[2][sl] + w[4][sl], 64)
        assert np.max(np.abs(An[i] - np.stack(ref))) <= 1e-10


def _steps(h, h0):
    return math.log(h / h0) / math.log(0.99)


def _opt_case(lb, m, resid_coef):
    ns = li.tgv_lattice(96, 80, m=m, h_over_s=2.8, jitter=0.3, seed=60 + m)
    h0 = 2.8 * ns.s
    xy, s, h0d = _dev(ns.xy), _dev(ns.s), _dev(h0)
    rp, col = lb.build_stencils(xy, h0d, ns.Lx, ns.Ly)
    hg, solves = lb.stencil_optimise(xy, h0d, s, ns.Lx, ns.Ly, rp, col, m, resid_coef=resid_coef)
    hg, solves = hg.cpu().numpy(), solves.cpu().numpy()
    assert np.all(hg <= h0) and np.all(solves >= 1)
    # every output is h0 times a whole number of 0.99 steps, taken by the same
    # repeated multiplication as the oracle's loop
    k = np.array([_steps(a, b) for a, b in zip(hg, h0)])
    assert np.all(np.abs(k - np.round(k)) < 1e-6)
    return ns, h0, rp.cpu().numpy(), col.cpu().numpy(), hg, solves


def _oracle_amax(ns, i, cand, m, h):
    """The oracle's largest amplitude response at stencil scale h (Section 4, steps 1-4)
    and cond_2(M_i) there."""
    dx0, dy0 = oracle.offsets(ns.xy, np.full(len(cand), i), cand, ns.Lx, ns.Ly)
    keep = dx0 * dx0 + dy0 * dy0 <= (2 * h) * (2 * h)
    dx, dy = dx0[keep], dy0[keep]
    W = oracle.abf_matrix(dx, dy, h, m)
    M = oracle.scaled_monomials(dx, dy, h, m).T @ W
    C = np.stack([oracle.selector(op, m, h) for op in ("x", "y", "L")], axis=1)
    psi, ok = oracle.lu_solve(M[None], C[None])
    assert ok[0]
    wts = W @ psi[0]
    amax = max(a.max() for a in oracle.amplitude_response(dx, dy, ns.s[i], wts[:, 0], wts[:, 1],
                                                          wts[:, 2], 16))
    return amax, np.linalg.cond(M)


@pytest.mark.parametrize("m", [4, 6, 8])
def test_stencil_optimise_matches_oracle_amplitude_test(lb, m):
    # with the residual test off, every stop is decided by the node count (exact on
    # both sides) or by an amplitude response against 1.01.  The responses agree to
    # rounding amplified by cond(M_i), so a node may stop one factor apart, but only
    # where the oracle's own response at the contested h lies within 1e-5 of the
    # bound, or where M_i is numerically singular there (cond > 1e14: a stencil with
    # exactly n nodes can reach 1e19, and then no two FP64 solvers agree on the
    # weights; the residual test exists to stop before such systems); everywhere
    # else h and the number of solves are identical
    ns, h0, rpn, coln, hg, solves = _opt_case(lb, m, math.inf)
    same = 0
    rows = np.random.default_rng(m).choice(ns.N, 48, replace=False)
    for i in rows:
        cand = coln[rpn[i]:rpn[i + 1]]
        hb, nsol = oracle.optimise_stencil_node(ns.xy, ns.s, i, cand, m, ns.Lx, ns.Ly, h0[i],
                                                resid_coef=math.inf)
        if hg[i] == hb and solves[i] == nsol:
            same += 1
            continue
        assert abs(round(_steps(hg[i], h0[i]) - _steps(hb, h0[i]))) == 1, (i, hg[i], hb)
        amax, cond = _oracle_amax(ns, i, cand, m, min(hg[i], hb))
        assert cond > 1e14 or abs(amax / 1.01 - 1.0) < 1e-5, (i, amax, cond)
    assert same >= len(rows) - 2, same


@pytest.mark.parametrize("m", [4, 6])
def test_stencil_optimise_with_residual_test_matches_oracle(lb, m):
    # alpha_L is a rounding-level quantity.  At the paper's coefficient (1e-4) its
    # bound sits inside the rounding noise of the solve over the whole range of h,
    # so the first h where the noise crosses it is solver-specific (Section 4 says
    # so; the oracle's own LU and LAPACK stop up to 5 factors apart on these nodes).
    # Ten times above that floor the test fires only at the conditioning cliff of
    # a too-small stencil, which every correct solver finds within a few factors
    # (the GPU's fused multiply-adds give a slightly smaller residual, so its stops
    # lean one factor later).
    ns, h0, rpn, coln, hg, solves = _opt_case(lb, m, 1e-3)
    diff = []
    for i in np.random.default_rng(m).choice(ns.N, 32, replace=False):
        cand = coln[rpn[i]:rpn[i + 1]]
        hb, _ = oracle.optimise_stencil_node(ns.xy, ns.s, i, cand, m, ns.Lx, ns.Ly, h0[i],
                                             resid_coef=1e-3)
        diff.append(round(_steps(hg[i], h0[i]) - _steps(hb, h0[i])))
    diff = np.array(diff)
    assert np.all(np.abs(diff) <= 4), diff
    assert np.mean(diff == 0) >= 0.5 and np.mean(np.abs(diff)) <= 1.0, diff


@pytest.mark.parametrize("m", [4, 6, 8])
def test_stencil_optimise_paper_coefficient_properties(lb, m):
    # at 1e-4 only what holds for any solver: outputs on the h0 0.99^k grid, at most
    # h0, and no further than the amplitude and node-count tests alone allow
    ns, h0, _, _, hg, _ = _opt_case(lb, m, 1e-4)
    _, _, _, _, h_amp, _ = _opt_case(lb, m, math.inf)
    assert np.all(hg >= h_amp)


def _oracle_tests_at(ns, i, cand, m, h):
    """Node count within 2h (the exact test of the neighbour search), and, if the
    count reaches n, the oracle's largest amplitude response and cond_2(M_i) at h."""
    dx0, dy0 = oracle.offsets(ns.xy, np.full(len(cand), i), cand, ns.Lx, ns.Ly)
    keep = dx0 * dx0 + dy0 * dy0 <= (2 * h) * (2 * h)
    count = int(np.sum(keep))
    if count < oracle.n_unknowns(m):
        return count, None, None
    dx, dy = dx0[keep], dy0[keep]
    W = oracle.abf_matrix(dx, dy, h, m)
    M = oracle.scaled_monomials(dx, dy, h, m).T @ W
    C = np.stack([oracle.selector(op, m, h) for op in ("x", "y", "L")], axis=1)
    psi, ok = oracle.lu_solve(M[None], C[None])
    if not ok[0]:  # singular for the oracle's LU as well
        return count, math.inf, math.inf
    wts = W @ psi[0]
    amax = max(a.max() for a in oracle.amplitude_response(dx, dy, ns.s[i], wts[:, 0], wts[:, 1],
                                                          wts[:, 2], 16))
    return count, amax, np.linalg.cond(M)


def _alpha0(m, h, coef=1e-4):
    n = oracle.n_unknowns(m)
    return coef * np.finfo(np.float64).eps * float(n) ** 4 / (h * m)


@pytest.mark.parametrize("m", [4, 6, 8])
def test_stencil_optimise_paper_coefficient_each_output_is_valid(lb, m):
    # At the paper's coefficient the residual test is decided by rounding noise, so
    # several outputs are correct; check that each sampled output is one of them,
    # using the GPU's own alpha_L (a solver-specific quantity) and the oracle for the
    # rest.  At the returned h every test passes: at least n nodes (exact), alpha_L
    # <= alpha_0, and the oracle's amplitude response <= 1.01.  At the next h
    # (0.99 h, one multiplication as in the loop) one test fails: fewer than n nodes,
    # alpha_L > alpha_0, an amplitude response above 1.01, a singular M_i, or the
    # iteration limit.  Amplitude decisions are contested only within 1e-5 of the
    # bound or where cond(M_i) > 1e14 (as in the test with the residual test off).
    ns = li.tgv_lattice(96, 80, m=m, h_over_s=2.8, jitter=0.3, seed=60 + m)
    h0 = 2.8 * ns.s
    xy, s, h0d = _dev(ns.xy), _dev(ns.s), _dev(h0)
    rp, col = lb.build_stencils(xy, h0d, ns.Lx, ns.Ly)
    hg, solves, alpha = lb.stencil_optimise(xy, h0d, s, ns.Lx, ns.Ly, rp, col, m, resid_coef=1e-4,
                                            alpha=True)
    hg, solves, alpha = hg.cpu().numpy(), solves.cpu().numpy(), alpha.cpu().numpy()
    rpn, coln = rp.cpu().numpy(), col.cpu().numpy()
    n = oracle.n_unknowns(m)

    def amp_fails(amax, cond):
        return amax > 1.01 or abs(amax / 1.01 - 1.0) < 1e-5 or cond > 1e14

    def amp_passes(amax, cond):
        return amax <= 1.01 or abs(amax / 1.01 - 1.0) < 1e-5 or cond > 1e14

    kinds = {}
    for i in np.random.default_rng(100 + m).choice(ns.N, 48, replace=False):
        cand = coln[rpn[i]:rpn[i + 1]]
        a_pass, a_stop = alpha[i]
        if np.isfinite(a_pass):  # the returned h passed every test
            count, amax, cond = _oracle_tests_at(ns, i, cand, m, hg[i])
            assert count >= n, (i, count)
            assert a_pass <= _alpha0(m, hg[i]), (i, a_pass)
            assert amp_passes(amax, cond), (i, amax, cond)
            h_next = hg[i] * 0.99
        else:  # nothing passed: h0 itself failed a test
            assert hg[i] == h0[i]
            h_next = h0[i]
        if solves[i] == 400:
            kinds["limit"] = kinds.get("limit", 0) + 1
            continue
        count, amax, cond = _oracle_tests_at(ns, i, cand, m, h_next)
        if count < n:
            assert np.isnan(a_stop)
            kind = "count"
        elif np.isfinite(a_stop) and a_stop > _alpha0(m, h_next):
            kind = "residual"
        elif np.isfinite(a_stop):
            assert amp_fails(amax, cond), (i, amax, cond)
            kind = "amplitude"
        else:  # a zero pivot on the GPU
            assert cond > 1e14, (i, cond)
            kind = "singular"
        kinds[kind] = kinds.get(kind, 0) + 1
    print(f"m = {m}: stops by", kinds)
    assert kinds.get("residual", 0) > 0  # the residual test takes part at this coefficient


def test_stencil_optimise_sixth_order_mean_matches_the_paper(lb):
    # Section 4: mean h/s about 1.5 for m = 6 when every node starts at 2.8 s
    ns = li.tgv_lattice(256, m=6, h_over_s=2.8, jitter=0.3, seed=3)
    h0 = 2.8 * ns.s
    xy, s, h0d = _dev(ns.xy), _dev(ns.s), _dev(h0)
    rp, col = lb.build_stencils(xy, h0d, ns.Lx, ns.Ly)
    hg, _ = lb.stencil_optimise(xy, h0d, s, ns.Lx, ns.Ly, rp, col, 6)
    ratio = (hg / s).cpu().numpy()
    assert 1.4 <= ratio.mean() <= 1.9, ratio.mean()
    # the optimised stencils still give a consistent operator; they end just above
    # the conditioning cliff (cond(M) up to ~1e8), so the reproduction residual is
    # cond(M) eps rather than the ~1e-12 of the h = 2.2 s stencils
    hs = hg * 1.0
    rp2, col2 = lb.build_stencils(xy, hs, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, hs, s, ns.Lx, ns.Ly, rp2, col2, 6, check=True)
    assert float(wb["residual"].max()) < 1e-6


def test_stencil_optimise_zero_iterations_returns_h0(lb):
    ns = li.tgv_lattice(20, m=4, h_over_s=2.8, jitter=0.3, seed=9)
    h0 = _dev(2.8 * ns.s)
    xy, s = _dev(ns.xy), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h0, ns.Lx, ns.Ly)
    hg, solves = lb.stencil_optimise(xy, h0, s, ns.Lx, ns.Ly, rp, col, 4, max_iter=0)
    assert torch.equal(hg, h0) and int(solves.max()) == 0
    with pytest.raises(lb.LabfmError):
        lb.stencil_optimise(xy, h0, s, ns.Lx, ns.Ly, rp, col, 5)
    with pytest.raises(lb.LabfmError):
        lb.stencil_optimise(xy, h0, s, ns.Lx, ns.Ly, rp, col, 4, factor=1.0)
