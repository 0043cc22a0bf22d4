"""The matrix-free right-hand side (each neighbour's weights recomputed from the
node's weight polynomials instead of read from a plan; the alternative the paper's
conclusions name for Lagrangian node sets) against the stored-weight path and the
oracle, FP64."""
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


def _case(lb, ns):
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wc = lb.weight_coefficients(xy, h, s, ns.Lx, ns.Ly, rp, col, ns.m, weights=True, check=True)
    return dict(ns=ns, xy=xy, h=h, s=s, rp=rp, col=col, wc=wc)


def _poly_weights(ns, rp, col, coef, m):
    """The weights the polynomials give, evaluated on the host: w^d_ji = psi P^d."""
    ex = [(p, q) for p in range(m + 1) for q in range(m + 1 - p)]  # idx(p, q) order
    w = np.zeros((6, len(col)))
    for i in range(ns.N):
        nb = col[rp[i]:rp[i + 1]]
        dx, dy = oracle.offsets(ns.xy, np.full(len(nb), i), nb, ns.Lx, ns.Ly)
        xh, yh = dx / ns.h[i], dy / ns.h[i]
        psi = oracle.wendland_c2(np.hypot(dx, dy) / ns.h[i])
        mono = np.stack([xh ** p * yh ** q for p, q in ex], axis=1)
        w[:, rp[i]:rp[i + 1]] = (mono @ coef[i]).T * psi
    return w


@pytest.mark.parametrize("m, nx, hs, jitter", [(4, 23, 1.7, 0.3), (6, 19, 2.2, 0.2), (8, 17, 2.8, 0.1),
                                               (10, 15, 3.3, 0.05)])
def test_polynomials_give_the_stored_and_the_oracle_weights(lb, m, nx, hs, jitter):
    ns = li.tgv_lattice(nx, nx + 3, m=m, h_over_s=hs, jitter=jitter, seed=m)
    c = _case(lb, ns)
    rp, col = c["rp"].cpu().numpy(), c["col"].cpu().numpy()
    coef = c["wc"]["coef"].cpu().numpy()
    assert coef.shape == (ns.N, (m + 1) * (m + 2) // 2, 6)
    wp = _poly_weights(ns, rp, col, coef, m)
    wg = c["wc"]["w"].cpu().numpy()
    ow = oracle.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, want_cond=True)
    n = oracle.n_unknowns(m)
    for i in range(ns.N):
        sl = slice(rp[i], rp[i + 1])
        scale = np.abs(wg[:, sl]).max(axis=1, keepdims=True)
        # the host evaluation of the same polynomials: rounding of the Horner sums
        assert (np.abs(wp[:, sl] - wg[:, sl]) / scale).max() <= 1e-11, i
        tol = max(50 * n * EPS64 * ow["cond1"][i], 1e-13)
        assert (np.abs(wp[:, sl] - ow["w"][:, sl]) / np.abs(ow["w"][:, sl]).max(axis=1, keepdims=True)).max() \
            <= tol + 1e-11, i


@pytest.mark.parametrize("m, nx, hs", [(4, 33, 1.7), (8, 29, 2.8), (10, 27, 3.3)])
def test_matrix_free_rhs_matches_stored_weights_and_oracle(lb, m, nx, hs):
    ns = li.tgv_lattice(nx, nx - 4, m=m, h_over_s=hs, jitter=0.2, seed=10 + m)
    c = _case(lb, ns)
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=4)
    phys = lb.Phys(100.0, 0.005, 0.2, -0.1)
    R = lb.rhs_matrix_free(c["xy"], c["h"], ns.Lx, ns.Ly, c["rp"], c["col"], m, c["wc"]["coef"], _dev(q),
                           phys).cpu().numpy()
    plan = lb.Plan(c["rp"], c["col"], c["wc"]["w"], c["wc"]["kappa"], c["s"], dtype=torch.float64)
    Rs = lb.rhs(plan, _dev(q), phys).cpu().numpy()
    plan.close()
    rp, col = c["rp"].cpu().numpy(), c["col"].cpu().numpy()
    Ro = oracle.rhs(q, c["wc"]["w"].cpu().numpy()[:5], rp, col, 100.0, 0.005, (0.2, -0.1))
    rel = lambda a, b: np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)  # noqa: E731
    assert np.all(rel(R, Rs) <= 1e-12), rel(R, Rs)
    assert np.all(rel(R, Ro) <= 1e-12), rel(R, Ro)


def test_matrix_free_rhs_full_size(lb):
    # the 512^2 m = 8 workload: the matrix-free right-hand side equals the stored
    # FP64 one at every node to 1e-12 (relative L2 per field)
    ns = li.tgv_lattice(512, m=8, h_over_s=2.8, jitter=0.3, seed=1)
    c = _case(lb, ns)
    q = _dev(li.tgv_fields(ns.xy, 10.0))
    phys = lb.Phys(100.0, 0.005)
    R = lb.rhs_matrix_free(c["xy"], c["h"], ns.Lx, ns.Ly, c["rp"], c["col"], 8, c["wc"]["coef"], q, phys)
    plan = lb.Plan(c["rp"], c["col"], c["wc"]["w"], c["wc"]["kappa"], c["s"], dtype=torch.float64)
    Rs = lb.rhs(plan, q, phys)
    plan.close()
    rel = ((R - Rs).norm(dim=1) / Rs.norm(dim=1)).cpu().numpy()
    assert np.all(rel <= 1e-12), rel


def test_matrix_free_arguments_are_checked(lb):
    ns = li.tgv_lattice(12, m=4, seed=2)
    c = _case(lb, ns)
    q = _dev(li.tgv_fields(ns.xy, 10.0))
    phys = lb.Phys(100.0, 0.005)
    with pytest.raises(lb.LabfmError):  # the output aliases the input
        lb.rhs_matrix_free(c["xy"], c["h"], ns.Lx, ns.Ly, c["rp"], c["col"], 4, c["wc"]["coef"], q, phys,
                           out=q)
    with pytest.raises(ValueError):  # coefficients of another order
        lb.rhs_matrix_free(c["xy"], c["h"], ns.Lx, ns.Ly, c["rp"], c["col"], 6, c["wc"]["coef"], q, phys)
    bad = c["col"].clone()
    bad[0] = ns.N
    with pytest.raises(lb.LabfmError):  # a malformed CSR
        lb.rhs_matrix_free(c["xy"], c["h"], ns.Lx, ns.Ly, c["rp"], bad, 4, c["wc"]["coef"], q, phys)
    # without stored weights (coefficients only) the build still gives kappa and status
    only = lb.weight_coefficients(c["xy"], c["h"], c["s"], ns.Lx, ns.Ly, c["rp"], c["col"], 4)
    assert torch.equal(only["coef"], c["wc"]["coef"]) and torch.equal(only["kappa"], c["wc"]["kappa"])
