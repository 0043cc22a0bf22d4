"""Pins of the oracle's modal (amplitude) response and stencil optimisation
(Sections 3 and 4): closed-form responses of classical central differences, the
stopping property of the h-reduction loop, and the paper's printed outcome."""
import math

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as o


def _unisolvent(offs, s, h, m):
    xy = np.vstack([[0.5, 0.5], 0.5 + s * np.asarray(offs, dtype=float)])
    N = xy.shape[0]
    rp = np.array([0, N - 1])
    col = np.arange(1, N, dtype=np.int32)
    out = o.build_weights(xy, np.full(N, h), np.full(N, s), rp, col, m, 1.0, 1.0,
                          periodic=(False, False), rows=np.array([0]))
    dx, dy = o.offsets(xy, np.zeros(N - 1, dtype=int), col, 1.0, 1.0, (False, False))
    return out["w"], dx, dy


def test_amplitude_response_of_second_order_stencil():
    s = 0.01
    w, dx, dy = _unisolvent([(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1)], s, s, 2)
    Ax, Ay, AL = o.amplitude_response(dx, dy, s, w[0], w[1], w[2] + w[4], nk=16)
    ks = np.pi / s * np.arange(1, 17) / 16
    assert np.allclose(Ax, np.sin(ks * s) / (ks * s), rtol=1e-9, atol=1e-12)
    assert np.allclose(Ay, np.sin(ks * s) / (ks * s), rtol=1e-9, atol=1e-12)
    assert np.allclose(AL, 2 * (1 - np.cos(ks * s)) / (ks * s) ** 2, rtol=1e-9, atol=1e-12)


def test_amplitude_response_of_fourth_order_stencil():
    s = 0.02
    offs = [(1, 0), (-1, 0), (2, 0), (-2, 0), (0, 1), (0, -1), (0, 2), (0, -2),
            (1, 1), (-1, 1), (1, -1), (-1, -1), (2, 1), (1, 2)]
    w, dx, dy = _unisolvent(offs, s, 1.2 * s, 4)
    Ax, Ay, AL = o.amplitude_response(dx, dy, s, w[0], w[1], w[2] + w[4], nk=16)
    ks = np.pi / s * np.arange(1, 17) / 16
    ref = (8 * np.sin(ks * s) - np.sin(2 * ks * s)) / (6 * ks * s)
    assert np.allclose(Ax, ref, rtol=1e-8, atol=1e-10)
    assert np.allclose(Ay, ref, rtol=1e-8, atol=1e-10)


def test_response_tends_to_one_at_low_wavenumber():
    ns = li.tgv_lattice(20, m=6, h_over_s=2.2, jitter=0.3, seed=4)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    w = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 6, ns.Lx, ns.Ly)["w"]
    A = o.modal_response(ns.xy, ns.s, rp, col, w, ns.Lx, ns.Ly, nk=64)
    # sixth-order consistent operators: the response at k = k_Ny / 64 is 1 to ~(k s)^6
    assert np.all(np.abs(A[:, :, 0] - 1.0) < 1e-6)


def _tests_pass(ns, i, cand, m, h, nk=16):
    """Both acceptance tests of Section 4 at stencil scale h (steps 1-4)."""
    n = o.n_unknowns(m)
    dx0, dy0 = o.offsets(ns.xy, np.full(len(cand), i), cand, ns.Lx, ns.Ly)
    keep = dx0 * dx0 + dy0 * dy0 <= (2 * h) * (2 * h)
    if keep.sum() < n:
        return False
    dx, dy = dx0[keep], dy0[keep]
    Xt = o.scaled_monomials(dx, dy, h, m)
    W = o.abf_matrix(dx, dy, h, m)
    M = Xt.T @ W
    C = np.stack([o.selector(op, m, h) for op in ("x", "y", "L")], axis=1)
    # the residual test is specific to the solver (Section 4 says so): near the
    # threshold LAPACK and the oracle's LU can decide differently, so the loop's
    # bookkeeping is checked with the same LU
    psi_b, ok = o.lu_solve(M[None], C[None])
    if not ok[0]:
        return False
    psi = psi_b[0]
    alpha = np.linalg.norm((M @ psi[:, 2] - C[:, 2]) * h * h)
    if alpha > 1e-4 * np.finfo(float).eps * n ** 4 / (h * m):
        return False
    wts = W @ psi
    A = o.amplitude_response(dx, dy, ns.s[i], wts[:, 0], wts[:, 1], wts[:, 2], nk)
    return max(a.max() for a in A) <= 1.01


@pytest.mark.parametrize("m", [4, 6])
def test_optimised_stencil_is_locally_minimal(m):
    """The result passes both tests (or is h0), and 1 % less would fail one of them."""
    ns = li.tgv_lattice(1024, m=m, h_over_s=2.8, jitter=0.3, seed=3)
    h0 = 2.8 * ns.s
    rows = np.random.default_rng(m).choice(ns.N, 6, replace=False)
    for i in rows:
        cand = o.neighbours_of(ns.xy, h0, i, ns.Lx, ns.Ly)
        hb, _ = o.optimise_stencil_node(ns.xy, ns.s, i, cand, m, ns.Lx, ns.Ly, h0[i])
        k = math.log(hb / h0[i]) / math.log(0.99)
        assert abs(k - round(k)) < 1e-6  # h0 times a whole number of 0.99 steps
        if hb < h0[i]:
            assert _tests_pass(ns, i, cand, m, hb)
        assert not _tests_pass(ns, i, cand, m, hb * 0.99)


def test_sixth_order_optimised_stencils_match_the_paper():
    # Section 4: for m = 6 the mean h/s drops to "approximately 1.5" (from 2.2; all
    # nodes start at 2.8 s).  The paper's node sets are additionally shifted toward
    # regularity, which allows somewhat smaller stencils than plain +-0.3 s jitter.
    ns = li.tgv_lattice(1024, m=6, h_over_s=2.8, jitter=0.3, seed=3)
    h0 = 2.8 * ns.s
    rows = np.random.default_rng(0).choice(ns.N, 24, replace=False)
    hs = []
    for i in rows:
        cand = o.neighbours_of(ns.xy, h0, i, ns.Lx, ns.Ly)
        hs.append(o.optimise_stencil_node(ns.xy, ns.s, i, cand, 6, ns.Lx, ns.Ly, h0[i])[0] / ns.s[i])
    assert 1.4 <= np.mean(hs) <= 1.9, np.mean(hs)


def test_amplitude_only_optimisation_is_solver_independent():
    """With the residual test off (resid_coef = inf) the loop stops on the node count
    or on a response against 1.01, so the oracle's LU and LAPACK agree exactly."""
    ns = li.tgv_lattice(96, 80, m=4, h_over_s=2.8, jitter=0.3, seed=64)
    h0 = 2.8 * ns.s
    rows = np.random.default_rng(4).choice(ns.N, 8, replace=False)
    lapack = lambda M, C: (np.linalg.solve(M, C), np.ones(M.shape[0], dtype=bool))
    for i in rows:
        cand = o.neighbours_of(ns.xy, h0, i, ns.Lx, ns.Ly)
        ha, na = o.optimise_stencil_node(ns.xy, ns.s, i, cand, 4, ns.Lx, ns.Ly, h0[i],
                                         resid_coef=math.inf)
        orig = o.lu_solve
        try:
            o.lu_solve = lapack
            hb, nb = o.optimise_stencil_node(ns.xy, ns.s, i, cand, 4, ns.Lx, ns.Ly, h0[i],
                                             resid_coef=math.inf)
        finally:
            o.lu_solve = orig
        assert ha == hb and na == nb
        assert ha < h0[i]
