"""Elementwise error budgets of the FP32 path against the FP64 oracle, derived
from the arithmetic (test infrastructure: used by the GPU tests, imports only
the oracle).

u = 2^-24 is the unit roundoff of float.  Inputs, stored weights and 1/s carry
a relative rounding of u each; a product or a sum adds u of its result.

Forward derivative (compensated sums, as the F32 kernels add the second
derivatives and the filter):
    B_d,i = 3 u sum_j |w_ji| (|phi_j| + |phi_i|) + 2 u |L_d,i|.

Right-hand side: the bounds above propagated linearly, with absolute values,
through eq. icns, plus 4 u times the absolute terms of each sum.

Right-hand-side adjoint Xbar = (dR/dq)^T m (pass A, then pass B, which adds
plain fused multiply-add chains without compensation):
  * derivative adjoints g (products of the node's own inputs): each carries at
    most (12 + |a|) u of its absolute terms (six input roundings, a float exp
    of 2 ulp whose argument a carries u |a|, the products and the scale s^-l);
  * own-value adjoints o (the node's derivative sums times m): the forward
    derivative budgets B times |m|, plus 8 u of the absolute terms (10 u + |a| u
    where nu = mu e^-a enters);
  * per stencil entry of the transposed operator: the weight (or its FP64
    combination, rounded once) carries 2 u, the gathered g its own error;
  * each accumulation chain of n fused multiply-adds adds at most n u of the sum
    of its absolute terms S (the standard recursive-summation bound); for node k
    the longest chain is 4 terms per transposed entry of one lane (4 ceil(t_k /
    4G) entries for t_k padded entries and G lanes per node), then log2 G
    shuffle adds and 8 operations of the own terms.
"""
import math

import numpy as np

from oracle import core as oracle

U32 = 2.0 ** -24


def deriv_bound(phi, w, rp, col):
    """Budget and value of L(phi)_i = sum_j (phi_j - phi_i) w_ji in FP32."""
    ri = oracle.row_index(rp)
    absum = np.bincount(ri, np.abs(w) * (np.abs(phi[col]) + np.abs(phi[ri])), minlength=len(rp) - 1)
    L = oracle.apply_op(phi, w, rp, col)
    return 3 * U32 * absum + 2 * U32 * np.abs(L), L


def derivative_bounds(q, w, rp, col):
    """(B, D): budgets and values of the twelve derivatives of eq. icns."""
    a, u, v = q
    B, D = {}, {}
    B["ax"], D["ax"] = deriv_bound(a, w[0], rp, col)
    B["ay"], D["ay"] = deriv_bound(a, w[1], rp, col)
    for name, f in (("u", u), ("v", v)):
        for k, op in enumerate(oracle.RHS_OPS):
            B[name + op], D[name + op] = deriv_bound(f, w[k], rp, col)
    return B, D


def rhs_bound(q, w, rp, col, c2, mu):
    a, u, v = q
    B, D = derivative_bounds(q, w, rp, col)
    nu = mu * np.exp(-a)
    ba = (np.abs(u) * B["ax"] + np.abs(v) * B["ay"] + B["ux"] + B["vy"]
          + 4 * U32 * (np.abs(u * D["ax"]) + np.abs(v * D["ay"]) + np.abs(D["ux"]) + np.abs(D["vy"])))
    out = [ba]
    for f, (x1, y1, a1, vis) in (("u", ("ux", "uy", "ax", ("uxx", "uyy", "vxy"))),
                                 ("v", ("vx", "vy", "ay", ("vyy", "vxx", "uxy")))):
        coef = (4.0 / 3.0, 1.0, 1.0 / 3.0)
        visc = sum(c * np.abs(D[n]) for c, n in zip(coef, vis))
        bvis = sum(c * B[n] for c, n in zip(coef, vis))
        b = (np.abs(u) * B[x1] + np.abs(v) * B[y1] + c2 * B[a1] + nu * bvis
             + 4 * U32 * (np.abs(u * D[x1]) + np.abs(v * D[y1]) + c2 * np.abs(D[a1]) + nu * visc))
        out.append(b)
    return np.stack(out)


def filter_bound(phi, phi_filtered, wf, rp, col):
    """phi + sum_j (phi_j - phi_i) kappa_i w^hyp_ji in FP32 (wf = kappa w^hyp per entry)."""
    b, _ = deriv_bound(phi, wf, rp, col)
    return b + 2 * U32 * np.abs(phi) + 2 * U32 * np.abs(phi_filtered)


def step_bound(q0, q1, dt, w, kappa, rp, col, c2, mu):
    """One FP32 time step from q0 (exact result q1): storage rounding of the state,
    dt sum_k |b_k| times the RHS budget at q0 (the stage states differ from q0 by
    O(dt), covered by a factor 2), and the filter budget at q1 (factor 2)."""
    B = rhs_bound(q0, w, rp, col, c2, mu)
    bsum = sum(abs(float(b)) for b in oracle.RK_B)
    wf = w[5] * np.repeat(kappa, np.diff(rp))
    out = []
    for f in range(3):
        bf, _ = deriv_bound(q1[f], wf, rp, col)
        out.append(8 * U32 * np.abs(q1[f]) + 2 * dt * bsum * B[f] + 2 * bf)
    return np.stack(out)


def _scatter(vals, col, N):
    return np.bincount(col, weights=vals, minlength=N)


def _chain_lengths(rp, col, N, G):
    """Longest fused multiply-add chain per node in the transposed gathers."""
    t = np.bincount(col, minlength=N)
    t_pad = (t + 3) // 4 * 4
    per_lane = 4 * np.ceil(t_pad / (4.0 * G))
    return 4 * per_lane + math.log2(G) + 8


def rhs_vjp_terms(q, m, w, rp, col, c2, mu):
    """The exact right-hand-side adjoint (dR/dq)^T m, the absolute sum S of its
    terms per node and field, and the budget's pieces."""
    a, u, v = q
    ma, mu_, mv = m
    N = q.shape[1]
    ri = oracle.row_index(rp)
    B, D = derivative_bounds(q, w, rp, col)
    nu = mu * np.exp(-a)
    t = 1.0 / 3.0
    ft = 4.0 / 3.0
    g = {"ax": -u * ma - c2 * mu_, "ay": -v * ma - c2 * mv, "ux": -ma - u * mu_, "uy": -v * mu_,
         "vx": -u * mv, "vy": -ma - v * mv,
         "uxx": ft * nu * mu_, "uyy": nu * mu_, "vxy": t * nu * mu_,
         "vxx": nu * mv, "vyy": ft * nu * mv, "uxy": t * nu * mv}
    gabs = {"ax": np.abs(u * ma) + c2 * np.abs(mu_), "ay": np.abs(v * ma) + c2 * np.abs(mv),
            "ux": np.abs(ma) + np.abs(u * mu_), "uy": np.abs(v * mu_), "vx": np.abs(u * mv),
            "vy": np.abs(ma) + np.abs(v * mv)}
    for k in ("uxx", "uyy", "vxy", "vxx", "vyy", "uxy"):
        gabs[k] = np.abs(g[k])
    dg = {k: (12.0 + np.abs(a)) * U32 * gabs[k] for k in g}
    # own-value adjoints and their budgets
    c6 = ft * D["uxx"] + D["uyy"] + t * D["vxy"]
    c7 = ft * D["vyy"] + D["vxx"] + t * D["uxy"]
    bc6 = ft * B["uxx"] + B["uyy"] + t * B["vxy"] + 4 * U32 * (ft * np.abs(D["uxx"]) + np.abs(D["uyy"])
                                                             + t * np.abs(D["vxy"]))
    bc7 = ft * B["vyy"] + B["vxx"] + t * B["uxy"] + 4 * U32 * (ft * np.abs(D["vyy"]) + np.abs(D["vxx"])
                                                             + t * np.abs(D["uxy"]))
    own = {"a": -nu * (c6 * mu_ + c7 * mv),
           "u": -(D["ax"] * ma + D["ux"] * mu_ + D["vx"] * mv),
           "v": -(D["ay"] * ma + D["uy"] * mu_ + D["vy"] * mv)}
    own_abs = {"a": nu * (np.abs(c6 * mu_) + np.abs(c7 * mv)),
               "u": np.abs(D["ax"] * ma) + np.abs(D["ux"] * mu_) + np.abs(D["vx"] * mv),
               "v": np.abs(D["ay"] * ma) + np.abs(D["uy"] * mu_) + np.abs(D["vy"] * mv)}
    own_err = {"a": nu * (bc6 * np.abs(mu_) + bc7 * np.abs(mv)) + (10.0 + np.abs(a)) * U32 * own_abs["a"],
               "u": B["ax"] * np.abs(ma) + B["ux"] * np.abs(mu_) + B["vx"] * np.abs(mv) + 8 * U32 * own_abs["u"],
               "v": B["ay"] * np.abs(ma) + B["uy"] * np.abs(mu_) + B["vy"] * np.abs(mv) + 8 * U32 * own_abs["v"]}
    ops = {"a": [("ax", 0), ("ay", 1)],
           "u": [("u" + op, k) for k, op in enumerate(oracle.RHS_OPS)],
           "v": [("v" + op, k) for k, op in enumerate(oracle.RHS_OPS)]}
    value, S, E0 = [], [], []
    for f in ("a", "u", "v"):
        val = own[f].copy()
        s_abs = own_abs[f].copy()
        err = own_err[f].copy()
        for name, k in ops[f]:
            wk = w[k]
            R = np.bincount(ri, weights=wk, minlength=N)
            Rabs = np.bincount(ri, weights=np.abs(wk), minlength=N)
            val += _scatter(wk * g[name][ri], col, N) - R * g[name]
            # absolute terms, with each g bounded by the sum of its own absolute
            # terms (so that S also bounds |dR/dq|^T |m| for a nonnegative m)
            s_abs += _scatter(np.abs(wk) * gabs[name][ri], col, N) + np.abs(R) * gabs[name]
            err += (_scatter(np.abs(wk) * (2 * U32 * np.abs(g[name][ri]) + dg[name][ri]), col, N)
                    + 2 * U32 * Rabs * np.abs(g[name]) + np.abs(R) * dg[name])
        value.append(val)
        S.append(s_abs)
        E0.append(err)
    return np.stack(value), np.stack(S), np.stack(E0)


def rhs_vjp_bound(q, m, w, rp, col, c2, mu, G=4):
    """Budget of the FP32 right-hand-side adjoint against the exact one."""
    _, S, E0 = rhs_vjp_terms(q, m, w, rp, col, c2, mu)
    n = _chain_lengths(rp, col, q.shape[1], G)
    return E0 + n * U32 * S


def filter_vjp_bound(lam, out, w_hyp, kappa, rp, col, G=4):
    """lam_k + sum_i kappa_i w^hyp_ik lam_i - (sum_j kappa_k w^hyp_kj) lam_k in FP32:
    weights kappa w rounded once (u) and inputs (u), plain chains of one FMA per
    transposed entry, the own term's row sum (2 u) and three more operations."""
    N = lam.shape[1]
    ri = oracle.row_index(rp)
    wf = w_hyp * kappa[ri]
    r = np.bincount(ri, weights=wf, minlength=N)
    rabs = np.bincount(ri, weights=np.abs(wf), minlength=N)
    t = np.bincount(col, minlength=N)
    chain = np.ceil(((t + 3) // 4 * 4) / (4.0 * G)) * 4 + math.log2(G) + 4
    bounds = []
    for f in range(3):
        terms = _scatter(np.abs(wf * lam[f][ri]), col, N)
        S = np.abs(lam[f]) + terms + np.abs(r * lam[f])
        bounds.append(3 * U32 * terms + 3 * U32 * rabs * np.abs(lam[f]) + chain * U32 * S
                      + 2 * U32 * np.abs(out[f]))
    return np.stack(bounds)


def step_vjp_bound(q, lam, lam_out, dt, w, kappa, rp, col, c2, mu, G=4):
    """One reverse time step in FP32 (labfm_rk_step_adjoint) against the exact one:
    the filter transpose's budget E_F, and the four stage adjoints, each at most
    dt |b_k| times the right-hand-side adjoint budget at the cotangent lam4 = Fil^T
    lam, plus the propagation of E_F through the transposed Jacobian (bounded by
    the absolute sums S at cotangent E_F), with the stage states taken as q (they
    differ by O(dt); factor 2, as for the forward step), and the storage rounding
    of the result."""
    lam4 = oracle.filter_vjp(lam, w[5], kappa, rp, col)
    EF = filter_vjp_bound(lam, lam4, w[5], kappa, rp, col, G)
    bsum = sum(abs(float(b)) for b in oracle.RK_B)
    _, S4, E4 = rhs_vjp_terms(q, lam4, w, rp, col, c2, mu)
    Ev = E4 + _chain_lengths(rp, col, q.shape[1], G) * U32 * S4
    _, Sprop, _ = rhs_vjp_terms(q, EF, w, rp, col, c2, mu)
    # the sweep's own additions and the stage cotangents dt (b Lambda + c Xbar)
    # round at most 8 u of the running cotangent; their rounding (3 u) reaches the
    # result through the transposed Jacobian like E_F
    return (8 * U32 * (np.abs(lam_out) + np.abs(lam4)) + EF
            + 2 * dt * bsum * (Ev + Sprop + 3 * U32 * S4))


# ---------------------------------------------------------------- boundaries (Section 7.1)

DERIVS = ("ax", "ay") + tuple(f + op for f in ("u", "v") for op in ("x", "y", "xx", "xy", "yy"))


def _node_rhs(kind, n, d, q, c, mu, g, target, L, mach, rho0, sigma):
    """(R_a, R_u, R_v) at one boundary node from its derivatives d and state q, as
    the oracle's boundary_rhs forms it (walls: the LODI wall with u held at zero)."""
    from oracle import boundary_oracle as bo
    if kind == bo.WALL:
        nx, ny = float(n[0]), float(n[1])
        rho = np.exp(q[0])
        a_xi = nx * d["ax"] + ny * d["ay"]
        du_xi = nx * (nx * d["ux"] + ny * d["uy"]) + ny * (nx * d["vx"] + ny * d["vy"])
        t = (-ny, nx)
        du_eta = t[0] * (t[0] * d["ux"] + t[1] * d["uy"]) + t[1] * (t[0] * d["vx"] + t[1] * d["vy"])
        Ra, _ = bo.wall_rhs(rho, c, c * c * rho * a_xi, du_xi, du_eta, nx * g[0] + ny * g[1])
        return np.array([Ra, 0.0, 0.0])
    return np.array(bo.open_boundary_rhs(kind, n, d, q, c, mu, g, target, L, mach, rho0, sigma))


def _abs_terms(kind, n, d, q, c, mu, g, target, L, mach, rho0, sigma):
    """S: the sum of the absolute values of the terms each boundary formula adds up
    (every product, relaxation and wave amplitude by its magnitude), per field.
    Frame components are bounded by the sums of the (x, y) components' magnitudes,
    and each viscous bracket (4/3 + 1 + 1/3 of frame second derivatives) by 8/3 of
    the summed magnitudes of both fields' Hessians."""
    from oracle import boundary_oracle as bo
    nx, ny = abs(float(n[0])), abs(float(n[1]))
    a, u, v = (float(x) for x in q)
    rho = np.exp(a)
    p = c * c * rho
    axi = nx * abs(d["ax"]) + ny * abs(d["ay"])
    aeta = ny * abs(d["ax"]) + nx * abs(d["ay"])
    uxi = nx * abs(u) + ny * abs(v)
    ueta = ny * abs(u) + nx * abs(v)
    grad = abs(d["ux"]) + abs(d["uy"]) + abs(d["vx"]) + abs(d["vy"])  # bounds every frame velocity derivative
    hess = sum(abs(d[f + "xx"]) + 2 * abs(d[f + "xy"]) + abs(d[f + "yy"]) for f in ("u", "v"))
    visc = 8.0 / 3.0 * hess
    L1 = 0.5 * (uxi + c) * (p * axi + rho * c * grad)
    if kind == bo.WALL:
        gn = nx * abs(g[0]) + ny * abs(g[1])
        return np.array([(2 * L1 + rho * c * gn) / (rho * c * c) + grad, 0.0, 0.0])
    T4 = 0.5 * (ueta * p * aeta + p * grad + rho * c * ueta * grad)
    V4 = 0.5 * mu * c * visc
    if kind == bo.OUTFLOW:
        L3 = uxi * grad
        L4 = sigma / (2 * L) * c * (1 - mach * mach) * (p + abs(target[0])) + (1 + mach) * T4 + V4
    else:
        T3 = ueta * grad + p * aeta / rho
        V3 = mu / rho * visc
        L3 = sigma * c / L * (ueta + abs(target[1])) + T3 + V3
        L4 = sigma * rho0 * c * c * (1 - mach * mach) / L * (uxi + abs(target[0])) + T4 + V4
    gsum = abs(g[0]) + abs(g[1])
    Sa = (L4 + L1) / (rho * c * c) + ueta * aeta + grad
    Sxi = (L4 + L1) / (rho * c) + ueta * grad + mu / rho * visc + gsum
    Seta = L3 + ueta * grad + p * aeta / rho + mu / rho * visc + gsum
    return np.array([Sa, nx * Sxi + ny * Seta, ny * Sxi + nx * Seta])


def boundary_rhs_bound(q, w, rp, col, bnd, c, mu, g=(0.0, 0.0), K=16):
    """Elementwise budget of one FP32 right-hand side of a domain with boundaries
    against the FP64 oracle (same weights).  Off the boundary nodes: rhs_bound (eq.
    icns) plus the body force's rounding.  At a boundary node (wall, inflow,
    outflow): the derivative budgets B_k propagated through the node's formula
    linearly, sum_k |dR/dd_k| B_k (the formulas are linear in each derivative, so
    central differences give these partials exactly up to rounding); the state's
    own rounding and the float exp (2 ulp, argument rounded), sum_f |dR/dq_f| (2 +
    |a|) u |q_f|; and K u S for the roundings inside the formula, S the sum of the
    absolute values of its terms and K = 16 the longest chain of operations through
    which one rounding can pass (frame rotation, wave amplitude, relaxation, the
    LODI combination and the rotation back)."""
    from oracle import boundary_oracle as bo
    B, D = derivative_bounds(q, w, rp, col)
    out = rhs_bound(q, w, rp, col, c * c, mu)
    out[1] += 4 * U32 * abs(g[0])
    out[2] += 4 * U32 * abs(g[1])
    sig = bnd.get("sigma", 0.278)
    for b, i in enumerate(bnd["nodes"]):
        kind = int(bnd["kind"][b])
        n = bnd["normal"][b]
        tgt = bnd["target"][b] if kind != bo.OUTFLOW else (bnd["target"][b][0], 0.0)
        tg = tgt[0] if kind == bo.OUTFLOW else tuple(tgt)
        d = {k: float(D[k][i]) for k in DERIVS}
        qi = q[:, i].astype(float)
        args = (c, mu, g, tg, bnd["L"], bnd["mach"], bnd["rho0"], sig)
        tot = np.zeros(3)
        for k in DERIVS:
            hk = 1e-6 * (abs(d[k]) + 1.0)
            dp, dm = dict(d), dict(d)
            dp[k] += hk
            dm[k] -= hk
            Jk = (_node_rhs(kind, n, dp, qi, *args) - _node_rhs(kind, n, dm, qi, *args)) / (2 * hk)
            tot += np.abs(Jk) * B[k][i]
        for f in range(3):
            hf = 1e-6 * (abs(qi[f]) + 1.0)
            qp, qm = qi.copy(), qi.copy()
            qp[f] += hf
            qm[f] -= hf
            Jf = (_node_rhs(kind, n, d, qp, *args) - _node_rhs(kind, n, d, qm, *args)) / (2 * hf)
            tot += np.abs(Jf) * (2.0 + abs(qi[0])) * U32 * abs(qi[f])
        S = _abs_terms(kind, n, d, qi, c, mu, g, tgt, bnd["L"], bnd["mach"], bnd["rho0"], sig)
        out[:, i] = tot + K * U32 * S
    return out


def boundary_step_bound(q0, q1, dt, w, kappa, rp, col, bnd, c, mu, g=(0.0, 0.0)):
    """One FP32 time step of a domain with boundaries from q0 (exact result q1): as
    step_bound, with boundary_rhs_bound for the right-hand side (the filter is off at
    the boundary nodes, kappa = 0 there)."""
    B = boundary_rhs_bound(q0, w, rp, col, bnd, c, mu, g)
    bsum = sum(abs(float(b)) for b in oracle.RK_B)
    wf = w[5] * np.repeat(kappa, np.diff(rp))
    out = []
    for f in range(3):
        bf, _ = deriv_bound(q1[f], wf, rp, col)
        out.append(8 * U32 * np.abs(q1[f]) + 2 * dt * bsum * B[f] + 2 * bf)
    return np.stack(out)
