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
