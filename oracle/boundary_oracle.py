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
    d[:, 0] -= ns.Lx * np.round(d[:, 0] / ns.Lx)  # minimum image in x
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

def channel_operator(ns, m: int = 4, m_wall: int = 4, h1d_over_s: float = 1.7):
    """Difference-form operators (row_ptr, col, w (6, nnz), kappa) for the node set of
    ``labfm_inputs.channel``, following the Table "Schemes for derivatives near
    boundaries":

    * interior and wall rows q = 3, 4: LABFM of order m (Sections 2, 3, 6) on the
      stencils |r_ji| <= 2 h_i inside the channel (periodic in x only);
    * rows q = 1, 2: d/dx, d/dy from ``strip_first_derivative_rows``; the second
      derivatives and the filter from LABFM of order m_wall on the same stencils;
    * wall nodes q = 0: d/dx, d/dy from ``strip_first_derivative_rows`` only (the
      velocity is held at zero there, the density follows eq. lodilnro), and
      kappa = 0: the wall node is not filtered (a reading: the paper lists
      "FD + 1D-LABFM" for its hyperviscous operator without the form of the mixed
      terms).
    """
    from . import labfm_oracle as core
    rp, col = core.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly, periodic=(True, False))
    per = (True, False)
    bw = core.build_weights(ns.xy, ns.h, ns.s, rp, col, m, ns.Lx, ns.Ly, periodic=per)
    bw4 = bw if m_wall == m else core.build_weights(ns.xy, ns.h, ns.s, rp, col, m_wall, ns.Lx, ns.Ly,
                                                    periodic=per)
    row = ns.meta["row"]
    N = ns.N
    entries, kappa = [], np.zeros(N)
    for i in range(N):
        a, b = rp[i], rp[i + 1]
        acc = {}
        if row[i] >= 3:
            if not bw["ok"][i]:
                raise ValueError(f"singular LABFM system at node {i}")
            for e in range(a, b):
                acc[int(col[e])] = bw["w"][:, e].copy()
            kappa[i] = bw["kappa"][i]
        else:
            if row[i] > 0:
                if not bw4["ok"][i]:
                    raise ValueError(f"singular LABFM system at node {i}")
                for e in range(a, b):
                    v = np.zeros(6)
                    v[2:] = bw4["w"][2:, e]
                    acc[int(col[e])] = v
                kappa[i] = bw4["kappa"][i]
            nodes, wx, wy = strip_first_derivative_rows(ns, i, 4, h1d_over_s)
            for j, ax, ay in zip(nodes, wx, wy):
                if j == i:
                    continue  # difference form: the node's own weight is -sum of the others
                v = acc.setdefault(int(j), np.zeros(6))
                v[0] += ax
                v[1] += ay
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
