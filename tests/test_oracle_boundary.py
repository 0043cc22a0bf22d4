"""Pins of the boundary operators of the oracle (Section 7.1 and Appendix A): the
five-point differences against the classical coefficient tables (Fornberg, Math.
Comp. 51 (1988)) and against exact differentiation of polynomials; one-dimensional
LABFM by exact reproduction of eta^k, k <= m, by its reduction to the central
differences on a uniform unisolvent row (independent of the RBF), by invariance to
the scale of psi, and by its convergence order; the rotation of Section 7.1 on
linear fields."""
from fractions import Fraction as F
from math import factorial

import numpy as np
import pytest

from oracle import boundary_oracle as bo
from oracle.labfm_oracle import wendland_c2

# classical five-point coefficients (units of s^-d), point offsets in increasing order
TABLES = {
    (bo.FD_CENTRAL, 1): [F(1, 12), F(-2, 3), F(0), F(2, 3), F(-1, 12)],
    (bo.FD_CENTRAL, 2): [F(-1, 12), F(4, 3), F(-5, 2), F(4, 3), F(-1, 12)],
    (bo.FD_ONE_SIDED, 1): [F(-25, 12), F(4), F(-3), F(4, 3), F(-1, 4)],
    (bo.FD_ONE_SIDED, 2): [F(35, 12), F(-26, 3), F(19, 2), F(-14, 3), F(11, 12)],
    (bo.FD_ASYMMETRIC, 1): [F(-1, 4), F(-5, 6), F(3, 2), F(-1, 2), F(1, 12)],
    (bo.FD_ASYMMETRIC, 2): [F(11, 12), F(-5, 3), F(1, 2), F(1, 3), F(-1, 12)],
}


@pytest.mark.parametrize("key", list(TABLES))
def test_five_point_differences_match_the_classical_tables(key):
    offsets, d = key
    assert bo.fd_weights(offsets, d) == TABLES[key]


@pytest.mark.parametrize("offsets", [bo.FD_ONE_SIDED, bo.FD_ASYMMETRIC, bo.FD_CENTRAL])
@pytest.mark.parametrize("d", [1, 2])
def test_five_point_differences_are_exact_on_quartics(offsets, d):
    # random quartic polynomials in exact rationals, differentiated at 0 with spacing s
    rng = np.random.default_rng(d + len(offsets))
    w = bo.fd_weights(offsets, d)
    for s in (F(1, 7), F(3, 2)):
        for _ in range(5):
            c = [F(int(v), 5) for v in rng.integers(-20, 20, size=5)]
            p = lambda x: sum(ck * x ** k for k, ck in enumerate(c))  # noqa: E731
            approx = sum(wq * p(q * s) for wq, q in zip(w, offsets)) / s ** d
            exact = factorial(d) * c[d]
            assert approx == exact
    # and not on every higher power: the first error term is q^5 (q^6 for the
    # symmetric central second difference, whose q^5 term cancels)
    x5, x6 = (sum(wq * F(q) ** k for wq, q in zip(w, offsets)) for k in (5, 6))
    assert x5 != 0 or x6 != 0
    if offsets == bo.FD_CENTRAL and d == 2:
        assert x5 == 0 and x6 != 0


def _row(n_side, s, jitter, seed):
    rng = np.random.default_rng(seed)
    q = np.arange(-n_side, n_side + 1, dtype=np.float64)
    eta = (q + rng.uniform(-jitter, jitter, size=q.size)) * s
    eta -= eta[n_side]  # node i at the origin
    return np.delete(eta, n_side)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_1d_labfm_reproduces_monomials_up_to_order_m(m):
    s = 0.01
    h = 1.3 * (m / 2 + 1) * s / 2  # support 2h spans ~m/2 + 1 nodes on each side
    eta = _row(m, s, 0.2, seed=m)
    eta = eta[np.abs(eta) <= 2 * h]
    we, wee, ok = bo.labfm_1d_weights(eta, h, m)
    assert ok and eta.size >= m
    for k in range(1, m + 1):
        phi = eta ** k / factorial(k)  # phi_i = 0 at the node
        scale = np.sum(np.abs(phi * we)) + 1.0
        assert abs(bo.apply_1d(0.0, phi, we) - (1.0 if k == 1 else 0.0)) <= 1e-9 * scale
        scale2 = np.sum(np.abs(phi * wee)) + 1.0
        assert abs(bo.apply_1d(0.0, phi, wee) - (1.0 if k == 2 else 0.0)) <= 1e-9 * scale2


@pytest.mark.parametrize("rbf", [wendland_c2, lambda q: np.where(q <= 2.0, 1.0, 0.0)],
                         ids=["wendland", "constant"])
def test_1d_labfm_on_a_uniform_unisolvent_row_is_the_central_difference(rbf):
    # m = 4 with the four nodes at -2s, -s, s, 2s: as many nodes as unknowns, so the
    # weights do not depend on the basis and equal the five-point central formulas
    s, h = 0.02, 0.021
    eta = np.array([-2.0, -1.0, 1.0, 2.0]) * s
    we, wee, ok = bo.labfm_1d_weights(eta, h, 4, rbf)
    assert ok
    c1 = [float(v) for v in TABLES[(bo.FD_CENTRAL, 1)]]
    c2 = [float(v) for v in TABLES[(bo.FD_CENTRAL, 2)]]
    np.testing.assert_allclose(we, np.array([c1[0], c1[1], c1[3], c1[4]]) / s, rtol=1e-9)
    np.testing.assert_allclose(wee, np.array([c2[0], c2[1], c2[3], c2[4]]) / s ** 2, rtol=1e-9)
    # the difference form puts -sum_j w_j on the node itself: the central -5/2
    assert abs(-np.sum(wee) * s ** 2 - float(c2[2])) < 1e-9


def test_1d_labfm_weights_do_not_depend_on_the_scale_of_psi():
    eta = _row(4, 0.01, 0.25, seed=5)
    h = 0.022
    eta = eta[np.abs(eta) <= 2 * h]
    a = bo.labfm_1d_weights(eta, h, 4)
    b = bo.labfm_1d_weights(eta, h, 4, lambda q: 7.5 * wendland_c2(q))
    np.testing.assert_allclose(a[0], b[0], rtol=1e-10)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-10)


@pytest.mark.parametrize("m", [2, 4])
def test_1d_labfm_converges_at_order_m(m):
    # derivative of sin(2 pi eta) at a node of a jittered row, spacing halved
    errs = []
    for s in (0.02, 0.01, 0.005):
        h = (m / 2 + 1.2) * s / 2
        eta = _row(m + 2, s, 0.2, seed=11)
        eta = eta[np.abs(eta) <= 2 * h]
        x0 = 0.137
        we, _, ok = bo.labfm_1d_weights(eta, h, m)
        assert ok
        approx = bo.apply_1d(np.sin(2 * np.pi * x0), np.sin(2 * np.pi * (x0 + eta)), we)
        errs.append(abs(approx - 2 * np.pi * np.cos(2 * np.pi * x0)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > m - 0.6), slopes


def test_rotation_from_boundary_coordinates():
    # phi = a x + b y: d/dxi = grad . n, d/deta = grad . t with t = (-n_y, n_x)
    rng = np.random.default_rng(2)
    for _ in range(10):
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        t = np.array([-n[1], n[0]])
        g = rng.standard_normal(2)
        dx, dy = bo.boundary_to_xy(n, g @ n, g @ t)
        assert abs(dx - g[0]) < 1e-14 and abs(dy - g[1]) < 1e-14


def test_hessian_rotation_from_boundary_coordinates():
    # the Hessian of a quadratic form in (x, y) seen in the boundary frame of any
    # normal (xi = r.n, eta = r.t): R H R^T with R's rows n and t; the rotation back
    # must return H
    rng = np.random.default_rng(5)
    for th in rng.uniform(0, 2 * np.pi, 16):
        n = np.array([np.cos(th), np.sin(th)])
        t = np.array([-n[1], n[0]])
        A = rng.standard_normal((2, 2))
        H = A + A.T
        R = np.stack([n, t])
        Hb = R @ H @ R.T
        got = bo.hessian_to_xy(n, Hb[0, 0], Hb[0, 1], Hb[1, 1])
        assert np.allclose(got, (H[0, 0], H[0, 1], H[1, 1]), rtol=0, atol=1e-13)


def _poly(c, x, y):
    # sum over i + j <= 4 of c[i, j] x^i y^j, and its x and y derivatives
    v = dx = dy = 0.0
    for i in range(5):
        for j in range(5 - i):
            v = v + c[i, j] * x ** i * y ** j
            if i:
                dx = dx + i * c[i, j] * x ** (i - 1) * y ** j
            if j:
                dy = dy + j * c[i, j] * x ** i * y ** (j - 1)
    return v, dx, dy


@pytest.mark.parametrize("q", [0, 1, 2])
def test_strip_first_derivatives_are_exact_on_quartics(q):
    # Section 7.1: five-point differences along the normal and 4th-order 1D LABFM
    # along the wall differentiate every polynomial of total degree <= 4 exactly,
    # on both walls (normals +y and -y)
    import labfm_inputs as li
    ns = li.channel(32, 14)
    rng = np.random.default_rng(q)
    c = rng.standard_normal((5, 5))
    meta = ns.meta
    nodes_q = np.flatnonzero((meta["row"] == q) & (np.abs(ns.xy[:, 0] - 0.5) < 0.2))
    assert nodes_q.size > 0 and set(meta["wall"][nodes_q]) == {0, 1}
    for i in nodes_q:
        nodes, wx, wy = bo.strip_first_derivative_rows(ns, int(i))
        # the polynomial about node i (unwrapped positions; no node crosses x = 0 or 1 here)
        d = ns.xy[nodes] - ns.xy[i]
        phi, _, _ = _poly(c, d[:, 0], d[:, 1])
        _, gx, gy = _poly(c, 0.0, 0.0)
        scale = np.sum(np.abs(wx * phi)) + np.sum(np.abs(wy * phi)) + 1.0
        assert abs(np.sum(wx * phi) - gx) <= 1e-11 * scale
        assert abs(np.sum(wy * phi) - gy) <= 1e-11 * scale


def _poly2(c, x, y):
    """sum c_ij x^i y^j (i + j <= 4) and its second derivatives xx, xy, yy."""
    v = dxx = dxy = dyy = 0.0
    for i in range(5):
        for j in range(5 - i):
            v = v + c[i, j] * x ** i * y ** j
            if i >= 2:
                dxx = dxx + i * (i - 1) * c[i, j] * x ** (i - 2) * y ** j
            if i and j:
                dxy = dxy + i * j * c[i, j] * x ** (i - 1) * y ** (j - 1)
            if j >= 2:
                dyy = dyy + j * (j - 1) * c[i, j] * x ** i * y ** (j - 2)
    return v, dxx, dxy, dyy


@pytest.mark.parametrize("kind", ["channel", "open_box"])
def test_boundary_node_second_derivatives_are_exact_on_quartics(kind):
    # "FD + 1D-LABFM" at a boundary node: the one-sided five-point second difference
    # along the normal column, 4th-order 1D LABFM along the boundary row, and the
    # normal difference of the rows' 1D-LABFM tangential derivative for the mixed
    # term, rotated to (x, y): exact on every polynomial of total degree <= 4, on
    # both boundaries of a channel (normals +-y) and of an open box (normals +-x)
    import labfm_inputs as li
    from oracle.labfm_oracle import minimum_image
    ns = li.channel(32, 14) if kind == "channel" else li.open_box(14, 32, jitter=0.1)
    per = (True, False) if kind == "channel" else (False, True)
    rng = np.random.default_rng(11)
    meta = ns.meta
    nodes0 = np.flatnonzero(meta["row"] == 0)
    assert set(meta["wall"][nodes0]) == {0, 1}
    for trial in range(3):
        c = rng.standard_normal((5, 5))
        for i in nodes0[::3]:
            w = bo.boundary_node_second_derivatives(ns, int(i))
            nodes = np.array(list(w))
            W = np.array([w[j] for j in nodes])  # (n, 3): xx, xy, yy
            assert np.all(np.abs(W.sum(axis=0)) <= 1e-9 * np.abs(W).sum(axis=0))
            dx = minimum_image(ns.xy[nodes, 0] - ns.xy[i, 0], ns.Lx, per[0])
            dy = minimum_image(ns.xy[nodes, 1] - ns.xy[i, 1], ns.Ly, per[1])
            phi = _poly2(c, dx, dy)[0]
            _, exx, exy, eyy = _poly2(c, 0.0, 0.0)
            got = W.T @ phi
            scale = np.abs(W).T @ np.abs(phi) + 1.0
            assert np.all(np.abs(got - (exx, exy, eyy)) <= 1e-10 * scale), (kind, i, got, (exx, exy, eyy))


def test_wall_keeps_a_hydrostatic_column_at_rest_with_the_consistent_wave():
    # a resting isothermal column under wall-normal gravity: dp/dxi = rho g.n.  With
    # L4 = L1 + rho c g.n the wall node's ln rho and u_xi stay put; with the printed
    # factor 2 ln rho drifts at -g.n / c
    c, rho = 10.0, 1.3
    for g_n in (-9.81, 0.7):
        dp = rho * g_n
        dl1, du1 = bo.wall_rhs(rho, c, dp, 0.0, 0.0, g_n, wall_factor=1.0)
        assert abs(dl1) < 1e-15 and abs(du1) < 1e-15
        dl2, _ = bo.wall_rhs(rho, c, dp, 0.0, 0.0, g_n, wall_factor=2.0)
        assert abs(dl2 + g_n / c) < 1e-14


def test_wall_without_gravity_reflects_acoustic_waves():
    # g = 0: L4 = L1, the incoming wave mirrors the outgoing one (perfect reflection),
    # and ln rho follows the compression -2 L1 / (rho c^2)
    c, rho = 10.0, 1.0
    dp, du = 0.3, -0.02
    L1, _, L4 = bo.wave_amplitudes(rho, c, 0.0, dp, du, 0.0)
    dl, dux = bo.wall_rhs(rho, c, dp, du, 0.0, 0.0)
    assert abs(dl - (-2 * L1 / (rho * c * c))) < 1e-15 and dux == 0.0
    # the outgoing amplitude at rest: L1 = -(c/2)(dp/dxi - rho c du/dxi)
    assert abs(L1 + 0.5 * c * (dp - rho * c * du)) < 1e-15


def _poiseuille_start_up(y, t, H, g, nu, nterms=400):
    # the channel started from rest under a constant body force g (x) between no-slip
    # walls: the sine series of the steady parabola decaying at the rates n^2 pi^2 nu / H^2
    u = g / (2 * nu) * y * (H - y)
    for k in range(nterms):
        n = 2 * k + 1
        u = u - (4 * g * H * H / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y / H)
                 * np.exp(-(n * np.pi) ** 2 * nu * t / H ** 2))
    return u


def _poiseuille_error(nx):
    # Section 8.2: Re = 10, Ma = 0.05, started from rest, velocity error at t U0 / H = 1
    import labfm_inputs as li
    from oracle import labfm_oracle as core
    ns = li.channel(nx, nx, m=6, jitter=0.1)
    H, U0 = ns.Ly, 1.0
    mu = U0 * H / 10.0
    g = 8 * mu * U0 / H ** 2
    c = U0 / 0.05
    op = bo.channel_operator(ns, 6, 4)
    q = np.zeros((3, ns.N))
    dt0 = core.stable_dt(np.stack([q[0], q[1] + U0, q[2]]), ns.s, c, mu)
    nsteps = int(np.ceil(1.0 / dt0))
    for _ in range(nsteps):
        q = bo.channel_time_step(q, 1.0 / nsteps, op, ns, c, mu, (g, 0.0))
    ua = _poiseuille_start_up(ns.xy[:, 1], 1.0, H, g, mu)
    assert np.all(q[1][ns.meta["row"] == 0] == 0.0) and np.all(q[2][ns.meta["row"] == 0] == 0.0)
    return np.linalg.norm(q[1] - ua) / np.linalg.norm(ua), float(np.abs(q[2]).max())


def test_poiseuille_start_up_converges_to_the_analytic_solution():
    # the transient is an exact solution of the isothermal equations (parallel flow,
    # uniform density): interior LABFM m = 6, the wall rows of Section 7.1, the no-slip
    # wall in LODI form.  The paper reports about 4th order at t* = 1
    e16, v16 = _poiseuille_error(16)
    e24, v24 = _poiseuille_error(24)
    order = np.log(e16 / e24) / np.log(24 / 16)
    assert e16 < 3e-3 and e24 < 4e-4, (e16, e24)
    assert order > 4.0, order
    # no cross-channel velocity develops beyond the discretisation error
    assert v16 < 1e-3 and v24 < 1e-3


def test_sampled_operator_rows_equal_the_full_operator():
    # channel_operator(rows=...) builds only the listed rows (for sampled checks of
    # large node sets): each equals the same row of the whole operator
    import labfm_inputs as li
    ns = li.channel(20, 18, m=6, jitter=0.1, seed=3)
    full = bo.channel_operator(ns, 6, 4)
    rows = np.array([0, 5, 17, 40, 77, 100, 200, ns.N - 1])
    sub = bo.channel_operator(ns, 6, 4, rows=rows)
    for k, i in enumerate(rows):
        a, b = slice(full[0][i], full[0][i + 1]), slice(sub[0][k], sub[0][k + 1])
        assert np.array_equal(full[1][a], sub[1][b])
        assert np.array_equal(full[2][:, a], sub[2][:, b])
        # kappa's F0 sum runs over each batch's padded stencil width (zeros added in
        # another order): equal to a few ulp
        assert abs(full[3][i] - sub[3][k]) <= 4 * np.finfo(float).eps * abs(full[3][i])
