"""Boundary operators of Section 7.1 and Appendix A (test infrastructure, like the
rest of this package: only tests may import it; nothing of the CUDA library).

* Differences along a boundary normal.  The weights of a difference formula over
  the points q s (q in a set of integer offsets) for the d-th derivative are the
  unique solution of the Taylor conditions

      sum_q w_q q^k / k! = [k == d],   k = 0 .. len(offsets) - 1,

  in units of s^-d: the definition of the formula of maximal order.  Section 7.1
  uses five points: one-sided (q = 0..4) at the wall node i0, asymmetric
  (q = -1..3) at i1 and central (q = -2..2) at i2.  Solved here in exact
  rational arithmetic.

* One-dimensional LABFM (Appendix A) for derivatives along the boundary tangent:
  monomials H_ji = [eta, eta^2/2, ..., eta^m/m!] (n = m), ABFs
  W^q_ji = psi(|eta_ji|/h_i) H_q(eta_ji/(h_i sqrt 2)) / sqrt(2^q), q = 1..m, with
  H_q the physicists' Hermite polynomial, M_i = sum_j H_ji (x) W_ji, M_i Psi^d = C^d
  with C^eta = e_1 and C^eta2 = e_2, and w^d_ji = W_ji . Psi^d.  The operator is the
  difference form sum_j (phi_j - phi_i) w^d_ji over the row's nodes j != i.

* The rotation of Section 7.1 from boundary coordinates (xi along the inward
  normal n, eta along the tangent) to (x, y).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

from .labfm_oracle import hermite, lu_solve, wendland_c2

FD_ONE_SIDED = (0, 1, 2, 3, 4)    # wall node i0
FD_ASYMMETRIC = (-1, 0, 1, 2, 3)  # first row in, i1
FD_CENTRAL = (-2, -1, 0, 1, 2)    # second row in, i2


def fd_weights(offsets, d: int) -> list[Fraction]:
    """Exact weights (units of s^-d) of the maximal-order difference formula for
    the d-th derivative over the points q s, q in `offsets` (Taylor conditions,
    solved by Gauss-Jordan elimination in rationals)."""
    q = [Fraction(v) for v in offsets]
    n = len(q)
    if not 0 <= d < n:
        raise ValueError("need 0 <= d < number of points")
    A = [[qq ** k / factorial(k) for qq in q] + [Fraction(int(k == d))] for k in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [A[r][n] for r in range(n)]


def labfm_1d_matrices(eta: np.ndarray, h: float, m: int, rbf=wendland_c2):
    """(H, W) for the offsets eta_ji of a boundary row (Appendix A): H[j, k] =
    eta_j^(k+1)/(k+1)!, W[j, q] = psi(|eta_j|/h) H_(q+1)(eta_j/(h sqrt 2))/sqrt(2^(q+1))."""
    eta = np.asarray(eta, dtype=np.float64)
    H = np.stack([eta ** k / factorial(k) for k in range(1, m + 1)], axis=1)
    psi = rbf(np.abs(eta) / h)
    z = eta / (h * np.sqrt(2.0))
    W = np.stack([psi * hermite(q, z) / np.sqrt(2.0 ** q) for q in range(1, m + 1)], axis=1)
    return H, W


def labfm_1d_weights(eta, h: float, m: int, rbf=wendland_c2):
    """Weights w^eta_j and w^eta2_j (Appendix A) for the offsets eta_j (j != i) of
    node i's boundary row; returns (w_eta, w_eta2, ok)."""
    H, W = labfm_1d_matrices(eta, h, m, rbf)
    M = H.T @ W  # M_kq = sum_j H_jk W_jq  (eq. disc_form1d)
    C = np.zeros((m, 2))
    C[0, 0] = 1.0  # C^eta
    if m >= 2:
        C[1, 1] = 1.0  # C^eta2
    psi, ok = lu_solve(M[None], C[None])
    w = W @ psi[0]
    return w[:, 0], w[:, 1], bool(ok[0])


def apply_1d(phi_i: float, phi_j: np.ndarray, w: np.ndarray) -> float:
    """The difference form sum_j (phi_j - phi_i) w_j."""
    return float(np.sum((np.asarray(phi_j, dtype=np.float64) - phi_i) * w))


def boundary_to_xy(n: np.ndarray, d_xi: np.ndarray, d_eta: np.ndarray):
    """(d/dx, d/dy) from (d/dxi, d/deta) with xi along the unit inward normal n and
    eta along the tangent t = (-n_y, n_x) (the rotation of Section 7.1)."""
    nx, ny = float(n[0]), float(n[1])
    return nx * d_xi - ny * d_eta, ny * d_xi + nx * d_eta


# --------------------------------------------------------------------------
# Section 7.1: first derivatives on the uniform rows along a wall
# --------------------------------------------------------------------------

_NORMAL_FD = {0: FD_ONE_SIDED, 1: FD_ASYMMETRIC, 2: FD_CENTRAL}


def strip_first_derivative_rows(ns, i: int, m1d: int = 4, h1d_over_s: float = 1.7, rbf=wendland_c2):
    """d/dx and d/dy at a node of the first three rows along a wall (row q = 0, 1, 2
    of ``labfm_inputs.channel``), as weights over nodes: the boundary-normal
    derivative by the five-point difference over the node's column (one-sided on
    the wall, asymmetric at q = 1, central at q = 2), the tangential one by
    one-dimensional LABFM of order m1d over the node's row (support 2 h, h =
    h1d_over_s s), both rotated to (x, y) (Table "Schemes for derivatives near
    boundaries").  Returns (nodes, w_x, w_y) with sum_j w_j phi_j the derivative
    (the node itself included)."""
    meta = ns.meta
    q = int(meta["row"][i])
    if q not in _NORMAL_FD:
        raise ValueError("strip rows 0, 1 and 2 only")
    wall, ix = meta["wall"][i], meta["column"][i]
    n = meta["normal"][i]
    s = float(ns.s[i])
    # the column: rows 0..4 of the same wall and x index, in order of distance
    col = np.array([int(np.flatnonzero((meta["wall"] == wall) & (meta["column"] == ix) &
                                       (meta["row"] == r))[0]) for r in range(5)])
    w_xi = np.array([float(v) for v in fd_weights(_NORMAL_FD[q], 1)]) / s
    # the row: same wall and row index, within 2h along the (periodic) tangent
    t = np.array([-n[1], n[0]])
    same = np.flatnonzero((meta["wall"] == wall) & (meta["row"] == q))
    same = same[same != i]
    d = ns.xy[same] - ns.xy[i]
    if ns.meta.get("kind") == "open_box":  # periodic in y
        d[:, 1] -= ns.Ly * np.round(d[:, 1] / ns.Ly)
    else:  # the channel: periodic in x
        d[:, 0] -= ns.Lx * np.round(d[:, 0] / ns.Lx)
    eta = d @ t
    h = h1d_over_s * s
    keep = np.abs(eta) <= 2 * h
    row_nodes, eta = same[keep], eta[keep]
    w_eta, _, ok = labfm_1d_weights(eta, h, m1d, rbf)
    if not ok:
        raise ValueError("singular one-dimensional system")
    nodes = np.concatenate([col, row_nodes, [i]])
    d_xi = np.concatenate([w_xi, np.zeros(row_nodes.size + 1)])
    d_eta = np.concatenate([np.zeros(5), w_eta, [-np.sum(w_eta)]])  # difference form
    wx, wy = boundary_to_xy(n, d_xi, d_eta)
    return nodes, wx, wy


def _column_and_row(ns, i):
    """Wall index, row q, column x-index and inward normal of a node of the five
    uniform rows, and the nodes of its normal column (rows 0..4)."""
    meta = ns.meta
    wall, ix, q = meta["wall"][i], meta["column"][i], int(meta["row"][i])
    col = np.array([int(np.flatnonzero((meta["wall"] == wall) & (meta["column"] == ix) &
                                       (meta["row"] == r))[0]) for r in range(5)])
    return wall, q, col, meta["normal"][i]


def _row_eta_weights(ns, k, h1d_over_s=1.7, rbf=wendland_c2):
    """1D LABFM (order 4, Appendix A) along the row of node k: its row neighbours
    within 2h and the weights of d/deta and d2/deta2 (difference form)."""
    meta = ns.meta
    n = meta["normal"][k]
    t = np.array([-n[1], n[0]])
    same = np.flatnonzero((meta["wall"] == meta["wall"][k]) & (meta["row"] == meta["row"][k]))
    same = same[same != k]
    d = ns.xy[same] - ns.xy[k]
    per_x = ns.meta.get("kind") != "open_box"  # the channel is periodic in x, the box in y
    if per_x:
        d[:, 0] -= ns.Lx * np.round(d[:, 0] / ns.Lx)
    else:
        d[:, 1] -= ns.Ly * np.round(d[:, 1] / ns.Ly)
    eta = d @ t
    h = h1d_over_s * float(ns.s[k])
    keep = np.abs(eta) <= 2 * h
    w1, w2, ok = labfm_1d_weights(eta[keep], h, 4, rbf)
    if not ok:
        raise ValueError("singular one-dimensional system")
    return same[keep], w1, w2


def boundary_node_second_derivatives(ns, i: int, h1d_over_s: float = 1.7):
    """Second derivatives at a boundary node i0 (row q = 0) from "FD + 1D-LABFM"
    (Table "Schemes for derivatives near boundaries"): d2/dxi2 by the one-sided
    five-point second difference along the normal column, d2/deta2 by 1D LABFM
    (C^eta2) along the boundary row, and the mixed d2/dxi deta (reading: the paper
    does not give its form) as the one-sided five-point first difference along the
    column of the rows' 1D LABFM d/deta (each column node's own row).  Rotated to
    (x, y) with d/dx = n_x d/dxi - n_y d/deta, d/dy = n_y d/dxi + n_x d/deta.
    Returns {node: (w_xx, w_xy, w_yy)} with sum_j w_j phi_j the derivative (the
    node itself included; the weights of each derivative sum to zero)."""
    _, q, col, n = _column_and_row(ns, i)
    if q != 0:
        raise ValueError("boundary nodes (row 0) only")
    s = float(ns.s[i])
    acc = {}

    def add(node, xixi, xieta, etaeta):
        v = acc.setdefault(int(node), np.zeros(3))
        v += (xixi, xieta, etaeta)

    w2 = [float(v) for v in fd_weights(FD_ONE_SIDED, 2)]
    w1 = [float(v) for v in fd_weights(FD_ONE_SIDED, 1)]
    for r in range(5):
        add(col[r], w2[r] / s ** 2, 0.0, 0.0)
    rows0, _, we2 = _row_eta_weights(ns, i, h1d_over_s)
    for j, w in zip(rows0, we2):
        add(j, 0.0, 0.0, w)
    add(i, 0.0, 0.0, -float(np.sum(we2)))
    for r in range(5):
        nbrs, we1, _ = _row_eta_weights(ns, col[r], h1d_over_s)
        c = w1[r] / s
        for j, w in zip(nbrs, we1):
            add(j, 0.0, c * w, 0.0)
        add(col[r], 0.0, -c * float(np.sum(we1)), 0.0)
    return {j: hessian_to_xy(n, a, b, c) for j, (a, b, c) in acc.items()}


def hessian_to_xy(n, d_xixi, d_xieta, d_etaeta):
    """Second derivatives in (x, y) from those in the boundary frame (xi along n, eta
    along t = (-n_y, n_x)): with x = n_x xi - n_y eta and y = n_y xi + n_x eta, the
    chain rule twice gives
        d_xx = n_x^2 d_xixi - 2 n_x n_y d_xieta + n_y^2 d_etaeta,
        d_xy = n_x n_y d_xixi + (n_x^2 - n_y^2) d_xieta - n_x n_y d_etaeta,
        d_yy = n_y^2 d_xixi + 2 n_x n_y d_xieta + n_x^2 d_etaeta."""
    nx, ny = float(n[0]), float(n[1])
    return (nx * nx * d_xixi - 2 * nx * ny * d_xieta + ny * ny * d_etaeta,
            nx * ny * d_xixi + (nx * nx - ny * ny) * d_xieta - nx * ny * d_etaeta,
            ny * ny * d_xixi + 2 * nx * ny * d_xieta + nx * nx * d_etaeta)


# --------------------------------------------------------------------------
# Section 7.1: the no-slip wall in the characteristic (LODI) form
# --------------------------------------------------------------------------

def wave_amplitudes(rho, c, u_xi, dp_dxi, du_xi_dxi, du_eta_dxi):
    """L1, L3 and L4 of eq. Ldef (L2 = 0 for isothermal flow)."""
    L1 = 0.5 * (u_xi - c) * (dp_dxi - rho * c * du_xi_dxi)
    L3 = u_xi * du_eta_dxi
    L4 = 0.5 * (u_xi + c) * (dp_dxi + rho * c * du_xi_dxi)
    return L1, L3, L4


def wall_rhs(rho, c, dp_dxi, du_xi_dxi, du_eta_deta, g_n, visc_xi=0.0, wall_factor=1.0):
    """d ln rho/dt (eq. lodilnro) and d u_xi/dt (eq. lodiu) at a no-slip wall node,
    u = 0, with L1 from eq. Ldef and the incoming wave set to L4 = L1 + f rho c g.n.
    The paper prints f = 2; with eq. lodiu only f = 1 holds u_xi at zero (its
    time derivative is -(L4 - L1)/(rho c) + visc_xi + g.n), which is the reading
    taken (wall_factor selects it).  visc_xi: the viscous term of eq. lodiu."""
    L1, _, _ = wave_amplitudes(rho, c, 0.0, dp_dxi, du_xi_dxi, 0.0)
    L4 = L1 + wall_factor * rho * c * g_n
    dlnrho = -(L4 + L1) / (rho * c * c) - du_eta_deta
    du_xi = -(L4 - L1) / (rho * c) + visc_xi + g_n
    return dlnrho, du_xi


# --------------------------------------------------------------------------
# Section 7.1: the channel (walls at y = 0 and H, periodic in x), all operators
# --------------------------------------------------------------------------

def channel_operator(ns, m: int = 4, m_wall: int = 4, h1d_over_s: float = 1.7, rows=None):
    """Difference-form operators (row_ptr, col, w (6, nnz), kappa) for the node set of
    ``labfm_inputs.channel``, following the Table "Schemes for derivatives near
    boundaries":

    * interior and wall rows q = 3, 4: LABFM of order m (Sections 2, 3, 6) on the
      stencils |r_ji| <= 2 h_i inside the channel (periodic in x only);
    * rows q = 1, 2: d/dx, d/dy from ``strip_first_derivative_rows``; the second
      derivatives and the filter from LABFM of order m_wall on the same stencils;
    * boundary nodes q = 0: d/dx, d/dy from ``strip_first_derivative_rows``, the
      second derivatives from ``boundary_node_second_derivatives`` ("FD +
      1D-LABFM"; a wall holds the velocity at zero and does not use them), and
      kappa = 0: the boundary node is not filtered (a reading: the paper lists
      "FD + 1D-LABFM" for its hyperviscous operator without its form).
    ``ns`` is a ``labfm_inputs.channel`` (periodic in x) or ``open_box`` (periodic
    in y) node set.  ``rows``: the operator rows of these nodes only (row_ptr over
    them, kappa per listed node), for sampled checks of large node sets.
    """
    from . import labfm_oracle as core
    per = (False, True) if ns.meta.get("kind") == "open_box" else (True, False)
    sel = np.arange(ns.N) if rows is None else np.asarray(rows, dtype=np.int64)
    rp, col = core.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=per, rows=sel)
    bw = core.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, periodic=per, rows=sel)
    bw4 = bw if m_wall == m else core.build_weights(ns.xy, ns.h, ns.s, rp, col, m_wall, ns.Lx, ns.Ly,
                                                    periodic=per, rows=sel)
    row = ns.meta["row"]
    N = len(sel)
    entries, kappa = [], np.zeros(N)
    for k, i in enumerate(sel):
        i = int(i)
        a, b = rp[k], rp[k + 1]
        acc = {}
        if row[i] >= 3:
            if not bw["ok"][k]:
                raise ValueError(f"singular LABFM system at node {i}")
            for e in range(a, b):
                acc[int(col[e])] = bw["w"][:, e].copy()
            kappa[k] = bw["kappa"][k]
        else:
            if row[i] > 0:
                if not bw4["ok"][k]:
                    raise ValueError(f"singular LABFM system at node {i}")
                for e in range(a, b):
                    v = np.zeros(6)
                    v[2:] = bw4["w"][2:, e]
                    acc[int(col[e])] = v
                kappa[k] = bw4["kappa"][k]
            nodes, wx, wy = strip_first_derivative_rows(ns, i, 4, h1d_over_s)
            for j, ax, ay in zip(nodes, wx, wy):
                if j == i:
                    continue  # difference form: the node's own weight is -sum of the others
                v = acc.setdefault(int(j), np.zeros(6))
                v[0] += ax
                v[1] += ay
            if row[i] == 0:
                for j, (bxx, bxy, byy) in boundary_node_second_derivatives(ns, i, h1d_over_s).items():
                    if j == i:
                        continue
                    v = acc.setdefault(int(j), np.zeros(6))
                    v[2] += bxx
                    v[3] += bxy
                    v[4] += byy
        entries.append(sorted(acc.items()))
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(e) for e in entries])
    cols = np.array([j for e in entries for j, _ in e], dtype=np.int64)
    w = np.array([v for e in entries for _, v in e]).T.reshape(6, -1)
    return row_ptr, cols, w, kappa


def channel_rhs(q, op, ns, c: float, mu: float, g=(0.0, 0.0)):
    """d/dt of (ln rho, u, v) in the channel: eq. icns at every node but the wall,
    where u = 0 is held (zero right-hand side for u, v) and ln rho follows
    eq. lodilnro through ``wall_rhs`` (wall-normal derivatives from the one-sided
    differences, the tangential one from 1D LABFM)."""
    from . import labfm_oracle as core
    row_ptr, col, w, _ = op
    R = core.rhs(q, w, row_ptr, col, c * c, mu, g)
    d = core.derivatives(q, w, row_ptr, col)
    wall = np.flatnonzero(ns.meta["row"] == 0)
    n = ns.meta["normal"][wall]
    t = np.stack([-n[:, 1], n[:, 0]], axis=1)
    a = q[0][wall]
    rho = np.exp(a)
    grad = lambda f: np.stack([d[f + "x"][wall], d[f + "y"][wall]], axis=1)  # noqa: E731
    ga, gu, gv = np.stack([d["ax"][wall], d["ay"][wall]], axis=1), grad("u"), grad("v")
    dn = lambda gr, vec: np.sum(gr * vec, axis=1)  # noqa: E731
    dlnrho_dxi = dn(ga, n)
    du_xi_dxi = n[:, 0] * dn(gu, n) + n[:, 1] * dn(gv, n)
    du_eta_deta = t[:, 0] * dn(gu, t) + t[:, 1] * dn(gv, t)
    g_n = n @ np.asarray(g, dtype=np.float64)
    Ra, _ = wall_rhs(rho, c, c * c * rho * dlnrho_dxi, du_xi_dxi, du_eta_deta, g_n)
    R[0][wall] = Ra
    R[1][wall] = 0.0
    R[2][wall] = 0.0
    return R


def channel_time_step(q, dt: float, op, ns, c: float, mu: float, g=(0.0, 0.0)):
    """One step in the channel: the four RK stages with ``channel_rhs``, then the
    filter (Section 6) with the operator's kappa (zero on the walls)."""
    from . import labfm_oracle as core
    row_ptr, col, w, kappa = op
    Q = core.rk_step(q, dt, lambda x: channel_rhs(x, op, ns, c, mu, g))
    return core.filter_fields(Q, w[5], kappa, row_ptr, col)


# --------------------------------------------------------------------------
# Section 7.1: outflow and inflow in the characteristic (LODI) form
# --------------------------------------------------------------------------

WALL, INFLOW, OUTFLOW = 0, 1, 2


def _boundary_frame(n, d, q):
    """The node's state and derivatives in the boundary frame (xi along the inward
    normal n, eta along t = (-n_y, n_x)), from the (x, y) derivatives d of
    ``labfm_oracle.derivatives`` at the node and its state q = (ln rho, u, v)."""
    nx, ny = float(n[0]), float(n[1])
    tx, ty = -ny, nx
    a, u, v = q

    def dxi(f):
        return nx * d[f + "x"] + ny * d[f + "y"]

    def deta(f):
        return tx * d[f + "x"] + ty * d[f + "y"]

    def hess(f, p, r):  # p . H(f) . r
        return (p[0] * r[0] * d[f + "xx"] + (p[0] * r[1] + p[1] * r[0]) * d[f + "xy"]
                + p[1] * r[1] * d[f + "yy"])

    N, T = (nx, ny), (tx, ty)
    fr = {"u_xi": nx * u + ny * v, "u_eta": tx * u + ty * v,
          "a_xi": dxi("a"), "a_eta": deta("a"),
          "uxi_xi": nx * dxi("u") + ny * dxi("v"), "uxi_eta": nx * deta("u") + ny * deta("v"),
          "ueta_xi": tx * dxi("u") + ty * dxi("v"), "ueta_eta": tx * deta("u") + ty * deta("v"),
          "uxi_xixi": nx * hess("u", N, N) + ny * hess("v", N, N),
          "uxi_etaeta": nx * hess("u", T, T) + ny * hess("v", T, T),
          "uxi_xieta": nx * hess("u", N, T) + ny * hess("v", N, T),
          "ueta_xixi": tx * hess("u", N, N) + ty * hess("v", N, N),
          "ueta_etaeta": tx * hess("u", T, T) + ty * hess("v", T, T),
          "ueta_xieta": tx * hess("u", N, T) + ty * hess("v", N, T)}
    return fr


def open_boundary_rhs(kind, n, d, q, c, mu, g, target, L, mach, rho0, sigma=0.278):
    """d/dt of (ln rho, u, v) at an outflow or inflow node (eq. lodi with L2 = 0 for
    isothermal flow), from the node's derivatives d (x, y components) and state q.
    Outgoing waves from eq. Ldef; the incoming ones:
      outflow (eq. outflowL): L4 = sigma/(2L) c (1 - M^2)(p - p_inf) + (1 - M) T4 + V4,
        T4 = -1/2 (u_eta dp/deta + p du_eta/deta + rho c u_eta du_xi/deta),
        V4 = mu c/2 (4/3 u_xi,xixi + u_xi,etaeta + 1/3 u_eta,xieta);  target = p_inf;
      inflow: L3 = sigma c/L (u_eta - u_eta,IN) + T3 + V3,
        L4 = sigma rho0 c^2 (1 - M^2)/L (u_xi - u_xi,IN) + T4 + V4,
        T3 = -(u_eta du_eta/deta + dp/deta / rho),
        V3 = mu/rho (4/3 u_eta,etaeta + u_eta,xixi + 1/3 u_xi,xieta);
        target = (u_xi,IN, u_eta,IN).
    (Reading: the paper prints the inflow's relaxations as (u_xi - u_xi,IN) in L3 and
    (u_eta - u_eta,IN) in L4; with eq. lodiu and eq. lodiv only L4 drives u_xi and
    L3 drives u_eta, so each relaxes its own component.)  The viscous conditions:
    at an outflow dtau_etaxi/deta = 0 drops that term from the viscous force of
    eq. lodiu, leaving dtau_xixi/dxi / mu = 4/3 u_xi,xixi - 2/3 u_eta,xieta; at an
    inflow dtau_etaeta/deta = 0 drops it from eq. lodiv, leaving dtau_etaxi/dxi / mu
    = u_eta,xixi + u_xi,xieta.  V3 and V4 keep the printed brackets.  Returns
    (R_a, R_u, R_v) in (x, y) components; g = (g_x, g_y)."""
    fr = _boundary_frame(n, d, q)
    nx, ny = float(n[0]), float(n[1])
    tx, ty = -ny, nx
    a = q[0]
    rho = np.exp(a)
    p = c * c * rho
    p_xi = c * c * rho * fr["a_xi"]
    p_eta = c * c * rho * fr["a_eta"]
    u_xi, u_eta = fr["u_xi"], fr["u_eta"]
    L1 = 0.5 * (u_xi - c) * (p_xi - rho * c * fr["uxi_xi"])
    visc_xi = 4.0 / 3.0 * fr["uxi_xixi"] + fr["uxi_etaeta"] + 1.0 / 3.0 * fr["ueta_xieta"]
    visc_eta = 4.0 / 3.0 * fr["ueta_etaeta"] + fr["ueta_xixi"] + 1.0 / 3.0 * fr["uxi_xieta"]
    T4 = -0.5 * (u_eta * p_eta + p * fr["ueta_eta"] + rho * c * u_eta * fr["uxi_eta"])
    V4 = 0.5 * mu * c * visc_xi
    if kind == OUTFLOW:
        p_inf = target
        L3 = u_xi * fr["ueta_xi"]
        L4 = sigma / (2.0 * L) * c * (1.0 - mach * mach) * (p - p_inf) + (1.0 - mach) * T4 + V4
        visc_xi_eq = 4.0 / 3.0 * fr["uxi_xixi"] - 2.0 / 3.0 * fr["ueta_xieta"]
        visc_eta_eq = visc_eta
    elif kind == INFLOW:
        uxi_in, ueta_in = target
        T3 = -(u_eta * fr["ueta_eta"] + p_eta / rho)
        V3 = mu / rho * visc_eta
        L3 = sigma * c / L * (u_eta - ueta_in) + T3 + V3
        L4 = sigma * rho0 * c * c * (1.0 - mach * mach) / L * (u_xi - uxi_in) + T4 + V4
        visc_xi_eq = visc_xi
        visc_eta_eq = fr["ueta_xixi"] + fr["uxi_xieta"]
    else:
        raise ValueError("kind must be INFLOW or OUTFLOW")
    g_xi = nx * g[0] + ny * g[1]
    g_eta = tx * g[0] + ty * g[1]
    Ra = -(L4 + L1) / (rho * c * c) - u_eta * fr["a_eta"] - fr["ueta_eta"]
    Rxi = -(L4 - L1) / (rho * c) - u_eta * fr["uxi_eta"] + mu / rho * visc_xi_eq + g_xi
    Reta = -L3 - u_eta * fr["ueta_eta"] - p_eta / rho + mu / rho * visc_eta_eq + g_eta
    return Ra, nx * Rxi + tx * Reta, ny * Rxi + ty * Reta


def boundary_rhs(q, op, bnd, c: float, mu: float, g=(0.0, 0.0)):
    """d/dt of (ln rho, u, v) in a domain with walls, inflows and outflows: eq. icns
    at every node but the boundary nodes, which follow ``wall_rhs`` (u held at zero)
    or ``open_boundary_rhs``.  bnd: dict with nodes, normal (n, 2), kind (WALL,
    INFLOW, OUTFLOW), target (n, 2: (u_xi,IN, u_eta,IN) for an inflow, p_inf in
    column 0 for an outflow) and the scalars L, mach, rho0, sigma."""
    from . import labfm_oracle as core
    row_ptr, col, w, _ = op
    R = core.rhs(q, w, row_ptr, col, c * c, mu, g)
    d = core.derivatives(q, w, row_ptr, col)
    for b, i in enumerate(bnd["nodes"]):
        n = bnd["normal"][b]
        di = {k: v[i] for k, v in d.items()}
        qi = q[:, i]
        kind = int(bnd["kind"][b])
        if kind == WALL:
            nx, ny = float(n[0]), float(n[1])
            rho = np.exp(qi[0])
            a_xi = nx * di["ax"] + ny * di["ay"]
            du_xi = nx * (nx * di["ux"] + ny * di["uy"]) + ny * (nx * di["vx"] + ny * di["vy"])
            t = (-ny, nx)
            du_eta = t[0] * (t[0] * di["ux"] + t[1] * di["uy"]) + t[1] * (t[0] * di["vx"] + t[1] * di["vy"])
            Ra, _ = wall_rhs(rho, c, c * c * rho * a_xi, du_xi, du_eta, nx * g[0] + ny * g[1])
            R[:, i] = (Ra, 0.0, 0.0)
        else:
            target = bnd["target"][b][0] if kind == OUTFLOW else tuple(bnd["target"][b])
            R[:, i] = open_boundary_rhs(kind, n, di, qi, c, mu, g, target, bnd["L"], bnd["mach"],
                                        bnd["rho0"], bnd.get("sigma", 0.278))
    return R


def boundary_time_step(q, dt: float, op, bnd, c: float, mu: float, g=(0.0, 0.0)):
    """One step with ``boundary_rhs``: the four RK stages, then the filter (Section 6)
    with the operator's kappa (zero on the boundary nodes)."""
    from . import labfm_oracle as core
    row_ptr, col, w, kappa = op
    Q = core.rk_step(q, dt, lambda x: boundary_rhs(x, op, bnd, c, mu, g))
    return core.filter_fields(Q, w[5], kappa, row_ptr, col)
