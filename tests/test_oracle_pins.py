"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each checks the oracle against
a printed value (tests/golden), a closed form, a textbook limit, an independent
library routine or an invariant, chosen so that a dropped term, a wrong sign,
index or operand anywhere in the oracle fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as o
from tests.conftest import golden


# ---------------------------------------------------------------- Section 2

def test_monomial_order_matches_printed_vector():
    rows = golden("monomial_order.txt")
    ex = o.monomial_exponents(4)
    for q, (a, b, den) in enumerate(rows):
        assert ex[q] == (int(a), int(b))
        assert math.factorial(int(a)) * math.factorial(int(b)) == int(den)
    # X ends with y^m / m!
    assert o.monomial_exponents(7)[-1] == (0, 7)


def test_n_unknowns_matches_formula_table():
    for m, n in golden("n_unknowns.txt"):
        assert o.n_unknowns(int(m)) == int(n) == len(o.monomial_exponents(int(m)))


def test_selectors_match_printed_vectors():
    for name, *vals in golden("selectors.txt"):
        c = o.selector(name, 4, 1.0)[:8]
        assert np.array_equal(c, np.array([float(v) for v in vals]))


def test_hyp_selector_is_expanded_power_of_laplacian():
    # (d_xx + d_yy)^2 = d_xxxx + 2 d_xxyy + d_yyyy  (Section 6, m = 4)
    ex = o.monomial_exponents(4)
    c = o.selector("hyp", 4, 1.0)
    want = {(4, 0): 1.0, (2, 2): 2.0, (0, 4): 1.0}
    for q, ab in enumerate(ex):
        assert c[q] == want.get(ab, 0.0)
    # scaling by H: entries of degree k carry h^-k
    assert np.allclose(o.selector("hyp", 4, 0.5), c * 0.5 ** -4)
    assert np.allclose(o.selector("x", 4, 0.5)[0], 2.0)


# ---------------------------------------------------------------- Section 3

def test_hermite_matches_rodrigues_formula():
    sp = pytest.importorskip("sympy")
    z = sp.Symbol("z")
    pts = np.array([-1.3, -0.4, 0.0, 0.7, 1.41])
    for a in range(11):
        expr = sp.simplify((-1) ** a * sp.exp(z ** 2) * sp.diff(sp.exp(-z ** 2), z, a))
        ref = np.array([float(expr.subs(z, float(p))) for p in pts])
        got = o.hermite(a, pts)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max())), a


def test_wendland_c2_is_the_textbook_function():
    # Wendland's C2 function for d <= 3 in the radius r = q/2: (1 - r)^4_+ (4 r + 1)
    q = np.linspace(0.0, 2.6, 53)
    r = q / 2.0
    ref = np.where(r < 1.0, (1.0 - r) ** 4 * (4.0 * r + 1.0), 0.0)
    assert np.allclose(o.wendland_c2(q), ref, rtol=1e-14, atol=1e-16)
    assert o.wendland_c2(np.array([0.0]))[0] == 1.0
    # C2 at the edge of the support: value and first two derivatives vanish at q = 2
    d = 1e-3
    assert abs(o.wendland_c2(np.array([2.0 - d]))[0]) < 10 * d ** 3


def test_rbf_scaling_does_not_change_weights():
    # w = W Psi with M Psi = C: any constant factor on psi cancels (Sections 2-3)
    ns = li.tgv_lattice(12, m=4, jitter=0.3, seed=5)
    rows = np.array([17, 70])
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    a = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 4, ns.Lx, ns.Ly, rows=rows)
    b = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 4, ns.Lx, ns.Ly, rows=rows,
                        rbf=lambda q: 7.5 * o.wendland_c2(q))
    assert np.allclose(a["w"], b["w"], rtol=1e-9, atol=1e-9 * np.abs(a["w"]).max())


@pytest.mark.parametrize("m", [4, 6, 8])
def test_h_scaling_leaves_the_solution_unchanged(m):
    # Section 2 (vector H): scaling the monomials and the selectors by powers of h
    # improves the conditioning of M but leaves the exact weights unchanged.  The
    # unscaled system (monomials x^a y^b / (a! b!) in physical units, selectors with
    # a unit entry at the derivative's position) solved by LAPACK gives the oracle's
    # weights to within the conditioning of both.  A jittered cloud with spacing
    # s = 0.6 keeps the unscaled system solvable at m = 8 while h^k still spans
    # more than a decade
    s0 = 0.6
    h0 = li.H_OVER_S[m] * s0
    rng = np.random.default_rng(40 + m)
    k = int(np.ceil(2 * h0 / s0)) + 1
    g = np.array([(i, j) for i in range(-k, k + 1) for j in range(-k, k + 1) if (i, j) != (0, 0)], dtype=float)
    offs = (g + rng.uniform(-0.2, 0.2, g.shape)) * s0
    offs = offs[np.hypot(offs[:, 0], offs[:, 1]) <= 2 * h0]
    xy = np.vstack([[50.0, 50.0], 50.0 + offs])
    N = xy.shape[0]
    rp = np.array([0, N - 1])
    col = np.arange(1, N, dtype=np.int32)
    ref = o.build_weights(xy, np.full(N, h0), np.full(N, s0), rp, col, m, 100.0, 100.0, rows=np.array([0]),
                          want_cond=True)
    ex = o.monomial_exponents(m)
    unit = {"x": [(1, 0)], "y": [(0, 1)], "xx": [(2, 0)], "xy": [(1, 1)], "yy": [(0, 2)]}
    dx, dy = offs[:, 0], offs[:, 1]
    X = np.stack([dx ** a * dy ** b / (math.factorial(a) * math.factorial(b)) for a, b in ex], axis=1)
    W = o.abf_matrix(dx, dy, h0, m)
    M = X.T @ W
    cond = max(np.linalg.cond(M, 1), ref["cond1"][0])
    assert cond < 1e12, cond  # the comparison is meaningful
    for d, op in enumerate(("x", "y", "xx", "xy", "yy")):
        C = np.array([1.0 if e in unit[op] else 0.0 for e in ex])
        w = W @ np.linalg.solve(M, C)
        got = ref["w"][d]
        err = np.abs(w - got).max() / np.abs(got).max()
        assert err <= max(1e-12, 100 * cond * np.finfo(float).eps), (m, op, err, cond)


@pytest.mark.parametrize("m", [4, 6, 8])
def test_weights_follow_the_lattice_symmetries(m):
    # on an unjittered lattice every stencil is symmetric under x -> -x, y -> -y and
    # x <-> y, so the weights must be: w^x odd in x and even in y, w^xx even in both,
    # w^xy odd in each, and w^x(dx, dy) = w^y(dy, dx), w^xx(dx, dy) = w^yy(dy, dx)
    ns = li.tgv_lattice(16, m=m, h_over_s=li.H_OVER_S[m], jitter=0.0, seed=0)
    rows = np.array([0, 77])
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    wb = o.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, rows=rows)
    for k, i in enumerate(rows):
        nb = col[rp[k]:rp[k + 1]]
        dx, dy = o.offsets(ns.xy, np.full(len(nb), i), nb, ns.Lx, ns.Ly)
        key = {(round(a / ns.s[i]), round(b / ns.s[i])): e for e, (a, b) in enumerate(zip(dx, dy))}
        w = wb["w"][:, rp[k]:rp[k + 1]]
        tol = 1e-9 * np.abs(w).max(axis=1)
        for (a, b), e in key.items():
            mx, my, sw = key[(-a, b)], key[(a, -b)], key[(b, a)]
            for d, (sx, sy) in enumerate(((-1, 1), (1, -1), (1, 1), (-1, -1), (1, 1))):
                assert abs(w[d, mx] - sx * w[d, e]) <= tol[d], (m, "x-mirror", d)
                assert abs(w[d, my] - sy * w[d, e]) <= tol[d], (m, "y-mirror", d)
            assert abs(w[0, sw] - w[1, e]) <= tol[0] and abs(w[2, sw] - w[4, e]) <= tol[2]
            assert abs(w[3, sw] - w[3, e]) <= tol[3]
            assert abs(w[5, mx] - w[5, e]) <= tol[5] and abs(w[5, sw] - w[5, e]) <= tol[5]


# --------------------------------------------- unisolvent stencils: classical FD

def _single_node_set(offs, s, h):
    xy = np.vstack([[0.5, 0.5], 0.5 + s * np.asarray(offs, dtype=float)])
    N = xy.shape[0]
    ns = li.NodeSet(xy, np.full(N, s), np.full(N, h), 1.0, 1.0, 0)
    rp = np.array([0, N - 1])
    col = np.arange(1, N, dtype=np.int32)
    return ns, rp, col


def _fd(name):
    for row in golden("central_fd.txt"):
        if row[0] == name:
            return [float(Fraction(v)) for v in row[1:]]
    raise KeyError(name)


@pytest.mark.parametrize("rbf", ["wendland", "constant"])
def test_unisolvent_m2_is_second_order_central_fd(rbf):
    s = 0.01
    offs = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1)]
    ns, rp, col = _single_node_set(offs, s, 1.0 * s)
    kw = {} if rbf == "wendland" else {"rbf": lambda q: np.where(q <= 2.0, 1.0, 0.0)}
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 2, 1.0, 1.0, periodic=(False, False),
                          rows=np.array([0]), **kw)
    assert out["ok"][0]
    w = out["w"]
    d1, d2 = _fd("d1_o2"), _fd("d2_o2")
    expect_x = np.array([d1[3], d1[1], 0, 0, 0]) / s
    expect_y = np.array([0, 0, d1[3], d1[1], 0]) / s
    expect_xx = np.array([d2[3], d2[1], 0, 0, 0]) / s ** 2
    expect_yy = np.array([0, 0, d2[3], d2[1], 0]) / s ** 2
    tol = 1e-9
    assert np.allclose(w[0], expect_x, atol=tol / s)
    assert np.allclose(w[1], expect_y, atol=tol / s)
    assert np.allclose(w[2], expect_xx, atol=tol / s ** 2)
    assert np.allclose(w[4], expect_yy, atol=tol / s ** 2)
    # difference form: the implied centre weight of the Laplacian is the classical -4/s^2
    assert np.isclose(-(w[2] + w[4]).sum(), 2 * d2[2] / s ** 2, rtol=1e-9)


@pytest.mark.parametrize("rbf", ["wendland", "constant"])
def test_unisolvent_m4_is_fourth_order_central_fd(rbf):
    s = 0.02
    offs = [(1, 0), (-1, 0), (2, 0), (-2, 0), (0, 1), (0, -1), (0, 2), (0, -2),
            (1, 1), (-1, 1), (1, -1), (-1, -1), (2, 1), (1, 2)]
    ns, rp, col = _single_node_set(offs, s, 1.2 * s)
    kw = {} if rbf == "wendland" else {"rbf": lambda q: np.where(q <= 2.0, 1.0, 0.0)}
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 4, 1.0, 1.0, periodic=(False, False),
                          rows=np.array([0]), **kw)
    assert out["ok"][0]
    w = out["w"]
    d1, d2 = _fd("d1_o4"), _fd("d2_o4")
    ex1 = np.zeros(14); ex1[[0, 1, 2, 3]] = [d1[3], d1[1], d1[4], d1[0]]
    ey1 = np.zeros(14); ey1[[4, 5, 6, 7]] = [d1[3], d1[1], d1[4], d1[0]]
    ex2 = np.zeros(14); ex2[[0, 1, 2, 3]] = [d2[3], d2[1], d2[4], d2[0]]
    ey2 = np.zeros(14); ey2[[4, 5, 6, 7]] = [d2[3], d2[1], d2[4], d2[0]]
    tol = 1e-8
    assert np.allclose(w[0] * s, ex1, atol=tol)
    assert np.allclose(w[1] * s, ey1, atol=tol)
    assert np.allclose(w[2] * s * s, ex2, atol=tol)
    assert np.allclose(w[4] * s * s, ey2, atol=tol)


# ---------------------------------------------------------------- reproduction

@pytest.mark.parametrize("m", [2, 4, 6, 8, 10])
def test_polynomial_reproduction(m):
    """sum_j X~_ji w_ji = C~^d for every monomial up to order m (eq. lsys).

    Checked per entry to 1e-10 relative to the magnitude of the summed terms
    (and never looser than 1e-10 absolute for the unit entries of C~)."""
    hs = {int(a): float(b) for a, b in golden("hs_convergence.txt")}[m]
    ns = li.tgv_lattice(20, m=m, h_over_s=hs, jitter=0.3, seed=11)
    rows = np.arange(0, ns.N, 37)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, rows=rows)
    assert out["ok"].all()
    ri = o.row_index(rp)
    gi = rows[ri]
    dx, dy = o.offsets(ns.xy, gi, col, ns.Lx, ns.Ly)
    hj = ns.h[gi]
    ex = o.monomial_exponents(m)
    lvec = {"x": 1, "y": 1, "xx": 2, "xy": 2, "yy": 2, "hyp": m}
    for d, op in enumerate(o.OPS):
        wt = out["w"][d] * hj ** lvec[op]
        C = o.selector(op, m, 1.0)
        for q, (a, b) in enumerate(ex):
            term = (dx / hj) ** a * (dy / hj) ** b / (math.factorial(a) * math.factorial(b)) * wt
            got = np.bincount(ri, term, minlength=len(rows))
            scale = np.maximum(np.bincount(ri, np.abs(term), minlength=len(rows)), 1.0)
            assert np.all(np.abs(got - C[q]) <= 1e-10 * scale), (op, a, b)


def _abf_matrix(dx, dy, h, m, x_scale=math.sqrt(2.0), rbf=None):
    """The ABFs of Section 3 built here from numpy's physicists' Hermite series:
    W^ab_j = psi(|r_j|/h) H_a(x_j/(h x_scale)) H_b(y_j/(h x_scale)), 1 <= a + b <= m,
    psi the Wendland C2 function (support 2h), one column per (a, b)."""
    from numpy.polynomial import hermite as H
    q = np.hypot(dx, dy) / h
    psi = np.where(q < 2.0, (1.0 - q / 2.0) ** 4 * (2.0 * q + 1.0), 0.0) if rbf is None else rbf(q)
    cols = []
    for k in range(1, m + 1):
        for b in range(k + 1):
            a = k - b
            ca = np.zeros(a + 1)
            ca[a] = 1.0
            cb = np.zeros(b + 1)
            cb[b] = 1.0
            cols.append(psi * H.hermval(dx / (h * x_scale), ca) * H.hermval(dy / (h * x_scale), cb))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("m", [4, 6, 8])
def test_weights_lie_in_the_span_of_the_hermite_wendland_abfs(m):
    """eq. w_abf: every weight vector of a node is a combination of its ABFs, which
    with the reproduction conditions (eq. lsys, pinned above) fixes the weights when a
    stencil has more nodes than unknowns.  The ABFs are built here independently of
    the oracle (numpy's Hermite series, the textbook Wendland function); ABFs with a
    planted mistake (the argument scaled by h instead of h sqrt 2, or another radial
    function) do not contain the oracle's weights."""
    hs = {int(a): float(b) for a, b in golden("hs_convergence.txt")}[m]
    ns = li.tgv_lattice(20, m=m, h_over_s=hs, jitter=0.3, seed=13)
    rows = np.arange(5, ns.N, 53)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, rows=rows)
    assert out["ok"].all()
    ri = o.row_index(rp)
    dx, dy = o.offsets(ns.xy, rows[ri], col, ns.Lx, ns.Ly)
    n = o.n_unknowns(m)

    def worst_residual(**abf):
        worst = 0.0
        for r, i in enumerate(rows):
            sl = slice(rp[r], rp[r + 1])
            A = _abf_matrix(dx[sl], dy[sl], ns.h[i], m, **abf)
            assert A.shape == (rp[r + 1] - rp[r], n) and A.shape[0] > n
            for d in range(len(o.OPS)):
                wv = out["w"][d][sl]
                coef, *_ = np.linalg.lstsq(A, wv, rcond=None)
                worst = max(worst, np.linalg.norm(A @ coef - wv) / np.linalg.norm(wv))
        return worst

    assert worst_residual() <= 1e-8
    assert worst_residual(x_scale=1.0) > 1e-3
    assert worst_residual(rbf=lambda q: np.where(q < 2.0, (1.0 - q / 2.0) ** 4, 0.0)) > 1e-3


def test_laplacian_is_sum_of_second_derivatives_on_test_function():
    # eq. p6 test function: the operator with C^L equals w^xx + w^yy (linearity of eq. lsys)
    ns = li.tgv_lattice(16, m=6, h_over_s=1.8, jitter=0.3, seed=3)
    rows = np.arange(0, ns.N, 29)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 6, ns.Lx, ns.Ly, rows=rows)
    ri = o.row_index(rp)
    gi = rows[ri]
    dx, dy = o.offsets(ns.xy, gi, col, ns.Lx, ns.Ly)
    W = o.abf_matrix(dx, dy, ns.h[gi], 6)
    # solve once more for C^L alone, node by node, and compare with w^xx + w^yy
    for k, i in enumerate(rows):
        sl = slice(rp[k], rp[k + 1])
        Xt = o.scaled_monomials(dx[sl], dy[sl], ns.h[i], 6)
        M = Xt.T @ W[sl]
        psi = np.linalg.solve(M, o.selector("L", 6, ns.h[i]))
        wl = W[sl] @ psi
        ref = out["w"][2][sl] + out["w"][4][sl]
        assert np.allclose(wl, ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


# ---------------------------------------------------------------- LU

def test_lu_matches_lapack_gesv():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 27, 27)) + 5 * np.eye(27)
    B = rng.standard_normal((20, 27, 6))
    X, ok = o.lu_solve(A, B)
    assert ok.all()
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-10, atol=1e-12)
    # a matrix that needs pivoting (zero leading entry)
    P = np.array([[[0.0, 1.0], [2.0, 3.0]]])
    X, ok = o.lu_solve(P, np.array([[[1.0], [5.0]]]))
    assert ok.all() and np.allclose(X[0, :, 0], [1.0, 1.0])
    # singular matrix is flagged, not returned as numbers
    S = np.array([[[1.0, 2.0], [2.0, 4.0]]])
    _, ok = o.lu_solve(S, np.ones((1, 2, 1)))
    assert not ok[0]


def test_lu_on_moment_matrices_matches_lapack():
    ns = li.tgv_lattice(16, m=8, h_over_s=2.8, jitter=0.3, seed=9)
    i = 40
    col = o.neighbours_of(ns.xy, ns.h, i, ns.Lx, ns.Ly)
    dx, dy = o.offsets(ns.xy, np.full(len(col), i), col, ns.Lx, ns.Ly)
    Xt = o.scaled_monomials(dx, dy, ns.h[i], 8)
    W = o.abf_matrix(dx, dy, ns.h[i], 8)
    M = Xt.T @ W
    C = np.stack([o.selector(op, 8, ns.h[i]) for op in o.OPS], axis=1)
    X, ok = o.lu_solve(M[None], C[None])
    ref = np.linalg.solve(M, C)
    assert ok[0]
    # agreement up to the conditioning of M
    err = np.abs(W @ X[0] - W @ ref).max(axis=0) / np.abs(W @ ref).max(axis=0)
    assert err.max() < 1e-16 * np.linalg.cond(M, 1) * 100


# ---------------------------------------------------------------- convergence

@pytest.mark.parametrize("m,nxs,nsamp", [(4, (16, 24, 32, 48), 300), (6, (16, 24, 32, 48, 64), 400),
                                        (8, (16, 24, 32, 48), 400), (10, (16, 20, 24, 32), 200)])
def test_convergence_slope_on_periodic_mode(m, nxs, nsamp):
    """Error of d/dx and the Laplacian of sin(2 pi x) cos(2 pi y) falls as s^m and
    s^(m-1) (Section 2: leading error O(h^(m+1-l)) at fixed h/s)."""
    hs = {int(a): float(b) for a, b in golden("hs_convergence.txt")}[m]
    eg, el = [], []
    for nx in nxs:
        ns = li.tgv_lattice(nx, m=m, h_over_s=hs, jitter=0.3, seed=7)
        rng = np.random.default_rng(1)
        rows = np.sort(rng.choice(ns.N, size=min(nsamp, ns.N), replace=False))
        rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
        out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, rows=rows)
        x, y = ns.xy[:, 0], ns.xy[:, 1]
        k = 2 * np.pi
        f = np.sin(k * x) * np.cos(k * y)
        ri = o.row_index(rp)
        gi = rows[ri]
        L = lambda d: np.bincount(ri, (f[col] - f[gi]) * out["w"][d], minlength=len(rows))
        fx = k * np.cos(k * x[rows]) * np.cos(k * y[rows])
        lap = -2 * k * k * f[rows]
        eg.append(np.sqrt(np.mean((L(0) - fx) ** 2)) / k)
        el.append(np.sqrt(np.mean((L(2) + L(4) - lap) ** 2)) / (2 * k * k))
    ls = np.log(1.0 / np.asarray(nxs, dtype=float))
    pg = np.polyfit(ls, np.log(eg), 1)[0]
    pl = np.polyfit(ls, np.log(el), 1)[0]
    assert pg >= m - 0.5, (pg, eg)
    assert pl >= m - 1.5, (pl, el)


# ---------------------------------------------------------------- stencil

def test_neighbours_match_kdtree_and_count():
    spatial = pytest.importorskip("scipy.spatial")
    ns = li.tgv_lattice(40, 36, m=8, h_over_s=2.8, jitter=0.3, seed=2)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    tree = spatial.cKDTree(ns.xy, boxsize=[ns.Lx, ns.Ly])
    r = 2.0 * ns.h[0]
    ref = tree.query_ball_point(ns.xy, r)
    for i in range(ns.N):
        got = set(col[rp[i]:rp[i + 1]].tolist())
        want = set(ref[i]) - {i}
        diff = got ^ want
        for j in diff:  # only pairs sitting on the radius to rounding may differ
            dx, dy = o.offsets(ns.xy, np.array([i]), np.array([j]), ns.Lx, ns.Ly)
            assert abs(math.hypot(dx[0], dy[0]) - r) < 1e-12
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    # N_i ~ 4 pi (h/s)^2 (Section 2)
    mean = rp[-1] / ns.N
    assert abs(mean / (4 * np.pi * 2.8 ** 2) - 1.0) < 0.03


def test_neighbours_inclusive_radius_and_no_self():
    xy = np.array([[0.1, 0.1], [0.3, 0.1], [0.1, 0.30000000000000004], [0.9, 0.1]])
    h = np.full(4, 0.1)
    rp, col = o.neighbours(xy, h, 1.0, 1.0)
    # node 1 at exactly 2h from node 0 is in; node 3 is 0.2 away through the periodic edge
    assert list(col[rp[0]:rp[1]]) == [1, 3]
    assert 0 not in col[rp[0]:rp[1]]


# ---------------------------------------------------------------- RK3(2)4[2R+]C

def test_rk_coefficients_satisfy_third_order_conditions():
    A = o.rk_butcher()
    b = list(o.RK_B)
    c = [sum(row) for row in A]
    # the published rationals approximate irrational exact values: in exact rational
    # arithmetic the four third-order conditions hold to ~1e-26, and a wrong digit
    # in any numerator or denominator would leave a residual above 1e-13
    tol = Fraction(1, 10 ** 20)
    assert abs(sum(b) - 1) < tol
    assert abs(sum(b[i] * c[i] for i in range(4)) - Fraction(1, 2)) < tol
    assert abs(sum(b[i] * c[i] ** 2 for i in range(4)) - Fraction(1, 3)) < tol
    assert abs(sum(b[i] * A[i][j] * c[j] for i in range(4) for j in range(4)) - Fraction(1, 6)) < tol
    # it is not fourth order (a 4-stage 3rd-order pair)
    assert sum(b[i] * c[i] ** 3 for i in range(4)) != Fraction(1, 4)


def test_rk_low_storage_update_is_third_order():
    # nonlinear autonomous system (a linear one would show the order of the
    # stability polynomial instead): y1' = -y1^2, y2' = y1 y2, exact
    # y1 = 1/(1 + t), y2 = 1 + t from y = (1, 1)
    f = lambda x: np.array([-x[0] * x[0], x[0] * x[1]])
    exact = np.array([0.5, 2.0])
    errs = []
    for n in (10, 20, 40):
        dt = 1.0 / n
        y = np.array([1.0, 1.0])
        for _ in range(n):
            y = o.rk_step(y, dt, f)
        errs.append(np.abs(y - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8) and np.all(rates < 3.4), rates


# ---------------------------------------------------------------- filter, dt

def test_filter_response_is_one_third_at_two_thirds_nyquist():
    """kappa_i makes (1 + kappa_i nabla^m) map the local mode cos(kx)cos(ky),
    k = 3 pi / (2 s_i), centred on node i, to 1/3 of itself at i (Section 6)."""
    ns = li.tgv_lattice(16, m=6, h_over_s=2.2, jitter=0.3, seed=4)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 6, ns.Lx, ns.Ly)
    for i in (0, 77, 200):
        k = 3 * np.pi / (2 * ns.s[i])
        dx, dy = o.offsets(ns.xy, np.full(ns.N, i), np.arange(ns.N), ns.Lx, ns.Ly)
        g = np.cos(k * dx) * np.cos(k * dy)
        f = o.filter_fields(np.stack([g, g, g]), out["w"][5], out["kappa"], rp, col)
        assert np.isclose(f[0][i], g[i] / 3.0, rtol=1e-9)
    # sign: kappa ~ -(-1)^(m/2) ... for m = 6 the continuous nabla^6 of the mode is
    # -(2k^2)^3 < 0, so F_0 > 0 and kappa > 0
    assert np.all(out["kappa"] > 0)


@pytest.mark.parametrize("m, hs", [(4, 1.7), (6, 2.2), (8, 2.8)])
def test_filter_is_a_contraction_on_a_uniform_lattice(m, hs):
    # Section 6: on a uniform lattice the filter 1 + kappa nabla^m is a symmetric
    # convolution that keeps constants (eigenvalue 1) and damps every other mode:
    # all eigenvalues of the filter matrix are real and in (-1, 1]; a wrong sign of
    # kappa or of the hyperviscous selector would push some above 1
    ns = li.tgv_lattice(16, m=m, h_over_s=hs, jitter=0.0, seed=0)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly)
    ri = o.row_index(rp)
    F = np.eye(ns.N)
    wf = out["w"][5] * out["kappa"][ri]
    np.add.at(F, (ri, col), wf)
    np.add.at(F, (ri, ri), -wf)
    ev = np.linalg.eigvals(F)
    assert np.abs(ev.imag).max() < 1e-10
    assert ev.real.max() <= 1.0 + 1e-12 and ev.real.min() > -1.0, (ev.real.min(), ev.real.max())
    assert np.sum(np.abs(ev.real - 1.0) < 1e-9) == 1  # only the constant mode is kept


def test_stable_dt_for_taylor_green():
    ns = li.tgv_lattice(64, m=4, jitter=0.0)
    q = li.tgv_fields(ns.xy, 10.0)
    dt = o.stable_dt(q, ns.s, 10.0, 0.005)
    # convective limit binds: s / (max|u| + c), max|u| <= 1 on the lattice
    s = 1.0 / 64
    assert s / 11.0 <= dt <= s / 10.0
    assert o.stable_dt(q, ns.s, 10.0, 1e3) < dt  # a large viscosity makes the viscous limit bind


def _dt_coefficients():
    d = {k: float(v) for k, v in golden("dt_coefficients.txt")}
    return d["convective"], d["viscous"]


def _one_node(a=0.0, u=0.0, v=0.0):
    return np.array([[a], [u], [v]], dtype=np.float64)


def test_stable_dt_viscous_branch_closed_form():
    # where the viscous limit binds, dt = C_visc s^2 rho / mu (eq. dt); each factor
    # is varied on its own so that a wrong coefficient, power of s, or dependence on
    # rho or mu fails
    _, cv = _dt_coefficients()
    c = 10.0
    base = o.stable_dt(_one_node(), np.array([0.01]), c, 10.0)
    assert base == pytest.approx(cv * 0.01 ** 2 * 1.0 / 10.0, rel=1e-15)
    assert o.stable_dt(_one_node(), np.array([0.02]), c, 10.0) == pytest.approx(4.0 * base, rel=1e-15)
    assert o.stable_dt(_one_node(a=np.log(3.0)), np.array([0.01]), c, 10.0) == pytest.approx(3.0 * base,
                                                                                               rel=1e-14)
    assert o.stable_dt(_one_node(), np.array([0.01]), c, 20.0) == pytest.approx(0.5 * base, rel=1e-15)
    # the velocity does not enter the viscous limit
    assert o.stable_dt(_one_node(u=0.3, v=-0.4), np.array([0.01]), c, 10.0) == pytest.approx(base, rel=1e-15)


def test_stable_dt_convective_branch_and_domain_minimum():
    cc, cv = _dt_coefficients()
    # |u| = 5 (3-4-5), c = 5, negligible viscosity: dt = C_conv s / (|u| + c)
    assert o.stable_dt(_one_node(u=3.0, v=4.0), np.array([0.01]), 5.0, 1e-12) == pytest.approx(
        cc * 0.01 / 10.0, rel=1e-15)
    # two nodes, one limited by each branch: the minimum over the domain of both
    q = np.array([[0.0, np.log(2.0)], [3.0, 0.0], [4.0, 0.0]])
    s = np.array([0.01, 0.004])
    mu = 0.05
    expect = min(cc * 0.01 / (5.0 + 5.0), cv * 0.004 ** 2 * 2.0 / mu,
                 cc * 0.004 / 5.0, cv * 0.01 ** 2 / mu)
    assert o.stable_dt(q, s, 5.0, mu) == pytest.approx(expect, rel=1e-15)
    assert expect == pytest.approx(cv * 0.004 ** 2 * 2.0 / mu, rel=1e-15)  # the viscous node binds


# ---------------------------------------------------------------- Navier-Stokes

def test_rhs_matches_tensor_form_of_the_equations():
    """eq. icns against eq. mass / eq. mom with tau = mu (grad u + grad u^T - 2/3 I div u),
    evaluated symbolically on a smooth compressible field (not divergence free)."""
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y")
    k = 2 * sp.pi
    a_e = sp.Rational(1, 50) * sp.sin(k * X) * sp.cos(2 * k * Y)
    u_e = sp.sin(k * X) + sp.Rational(1, 2) * sp.cos(k * Y)
    v_e = sp.Rational(1, 3) * sp.cos(k * X) * sp.sin(k * Y) + sp.Rational(1, 4) * sp.sin(k * X)
    c2, mu, gx, gy = 100.0, 0.01, 0.3, -0.2
    rho = sp.exp(a_e)
    p = c2 * rho
    U = sp.Matrix([u_e, v_e])
    grad = lambda f: sp.Matrix([sp.diff(f, X), sp.diff(f, Y)])
    gu = sp.Matrix([[sp.diff(u_e, X), sp.diff(u_e, Y)], [sp.diff(v_e, X), sp.diff(v_e, Y)]])
    div = sp.diff(u_e, X) + sp.diff(v_e, Y)
    tau = mu * (gu + gu.T - sp.Rational(2, 3) * sp.eye(2) * div)
    divtau = sp.Matrix([sp.diff(tau[0, 0], X) + sp.diff(tau[0, 1], Y),
                        sp.diff(tau[1, 0], X) + sp.diff(tau[1, 1], Y)])
    ra = -(U.dot(grad(a_e))) - div
    rmom = -(gu * U) - grad(p) / rho + divtau / rho + sp.Matrix([gx, gy])
    f_ra = sp.lambdify((X, Y), ra, "numpy")
    f_ru = sp.lambdify((X, Y), rmom[0], "numpy")
    f_rv = sp.lambdify((X, Y), rmom[1], "numpy")
    fa, fu, fv = (sp.lambdify((X, Y), e, "numpy") for e in (a_e, u_e, v_e))

    ns = li.tgv_lattice(40, m=8, h_over_s=2.8, jitter=0.3, seed=6)
    rows = np.arange(0, ns.N, 13)
    rp_r, col_r = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, rows=rows)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp_r, col_r, 8, ns.Lx, ns.Ly, rows=rows)
    # evaluate the oracle RHS only at the sampled rows: embed them in a full CSR
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    cnt = np.zeros(ns.N, dtype=np.int64)
    cnt[rows] = np.diff(rp_r)
    rp[1:] = np.cumsum(cnt)
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    q = np.stack([fa(x, y) * np.ones_like(x), fu(x, y), fv(x, y)])
    R = o.rhs(q, out["w"][:5], rp, col_r, c2, mu, (gx, gy))
    xr, yr = x[rows], y[rows]
    ref = [f_ra(xr, yr), f_ru(xr, yr), f_rv(xr, yr)]
    for fld in range(3):
        err = np.abs(R[fld][rows] - ref[fld]).max() / np.abs(ref[fld]).max()
        assert err < 2e-4, (fld, err)


def test_taylor_green_decay_rate():
    """Kinetic energy of the Taylor-Green vortex decays as e^(2bt),
    b = -8 pi^2 H / (2 Re) (Section 8.1), at low Mach number."""
    b = float(dict(golden("taylor_green.txt"))["b"])
    mu = float(dict(golden("taylor_green.txt"))["mu"])
    ns = li.tgv_lattice(32, m=8, h_over_s=2.8, jitter=0.1, seed=1)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 8, ns.Lx, ns.Ly)
    c = 10.0
    q = li.tgv_fields(ns.xy, c)
    dt = o.stable_dt(q, ns.s, c, mu)
    ts, ke = [0.0], [o.kinetic_energy(q, ns.s)]
    for k in range(60):
        q = o.time_step(q, dt, out["w"], out["kappa"], rp, col, c * c, mu)
        ts.append((k + 1) * dt)
        ke.append(o.kinetic_energy(q, ns.s))
    rate = np.polyfit(ts, np.log(ke), 1)[0]
    assert abs(rate / (2 * b) - 1.0) < 0.02, rate
