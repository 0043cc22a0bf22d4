"""Section 8.3's Lamb-Oseen vortex study on the GPU, shared by the GPU test and the
benchmark's ``--only lamb_oseen`` leg: a vortex on a uniform stream (Ma = 0.05,
R_c = H/25, C = c H/300, Re = 7500) in the unit box with the inflow at x = 0, the
outflow at x = H and periodic y; LABFM m = 6 inside, m = 4 on the boundary rows'
second derivatives; the L2 norm of the disturbance u* = (u - U0, v)/U0 sampled in
t* = t U0 / R_c, and its convergence towards the finest resolution.

Readings (the paper gives no more): the node disorder is the jittered lattice of
``labfm_inputs.open_box`` at +-0.05 s (the paper's own generator of Section 5 is
not reproduced); the L2 norm is the node-volume weighted mean square over the box,
sqrt(sum_i s_i^2 |u*_i|^2 / H^2); the error of a resolution is the root mean square
over the sampled times of its norm minus the finest one's; the NSCBC length L is the
box length H and p_inf = rho0 c^2."""
import time

import numpy as np

import labfm_inputs as li
from tests.conftest import golden

U0, RHO0 = 1.0, 1.0


def printed():
    g = {r[0]: [float(v) for v in r[1:]] for r in golden("lamb_oseen.txt")}
    return [int(v) for v in g["resolution"]], g["rate"]


def sigma():
    return {k: float(v) for k, v in golden("nscbc.txt")}["sigma"]


def run(lb, torch, r_over_s: int, t_end: float = 20.0, sample: float = 0.1, m: int = 6, m_wall: int = 4,
        jitter: float = 0.05, dtype=None, seed: int = 0) -> dict:
    """One resolution: returns t*, the disturbance norm at each sampled t*, the step
    count and the timings."""
    dtype = torch.float64 if dtype is None else dtype
    n = int(round(r_over_s / li.LAMB_OSEEN_RC_OVER_H))   # H / s
    ns = li.open_box(n, n, m=m, jitter=jitter, seed=seed)
    H = ns.Ly
    Rc = li.LAMB_OSEEN_RC_OVER_H * H
    c = U0 / li.LAMB_OSEEN_MACH
    mu = U0 * Rc * RHO0 / li.LAMB_OSEEN_RE
    cols, normals = li.channel_walls(ns)
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    xy, h, s = dev(ns.xy), dev(ns.h), dev(ns.s)
    t0 = time.perf_counter()
    op = lb.build_wall_operator(xy, h, s, ns.Lx, ns.Ly, m, m_wall, dev(cols, torch.int32), dev(normals), 1.7,
                                periodic=(False, True), check=True)
    if op["n_failed"]:
        raise RuntimeError(f"{op['n_failed']} singular LABFM systems at R_c/s = {r_over_s}")
    plan = lb.Plan(op["row_ptr"], op["col"], op["w"], op["kappa"], s, dtype=dtype)
    n_b = cols.shape[0] // 2
    kind = np.array([lb.INFLOW] * n_b + [lb.OUTFLOW] * n_b, dtype=np.int32)
    target = np.zeros((2 * n_b, 2))
    target[:n_b, 0] = U0                   # inflow: (u_xi, u_eta) = (U0, 0), xi = +x
    target[n_b:, 0] = RHO0 * c * c         # outflow: p_inf
    plan.set_boundaries(dev(cols[:, 0], torch.int32), dev(normals), dev(kind, torch.int32), dev(target),
                        sigma=sigma(), L=ns.Lx, mach=li.LAMB_OSEEN_MACH, rho0=RHO0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Q = dev(li.lamb_oseen_fields(ns.xy, c, U0=U0, H=H, rho0=RHO0, centre=(0.5 * ns.Lx, 0.5 * H)), dtype)
    dt0 = float(lb.stable_dt(plan, Q, s, c, mu).item())
    tau = sample * Rc / U0
    k = int(np.ceil(tau / dt0))
    dt = tau / k
    vol = (s * s / (ns.Lx * H)).to(dtype)
    phys = lb.Phys(c * c, mu)
    work = lb.workspace(plan)

    def norm():
        du = (Q[1] - U0) / U0
        dv = Q[2] / U0
        return torch.sqrt(torch.sum(vol * (du * du + dv * dv)))

    nsamp = int(round(t_end / sample))
    norms = torch.empty(nsamp + 1, dtype=torch.float64, device="cuda")
    norms[0] = norm()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for j in range(nsamp):
        lb.rk_step(plan, Q, dt, k, phys, work=work)
        norms[j + 1] = norm()
    ev1.record()
    torch.cuda.synchronize()
    out = {"r_over_s": r_over_s, "nodes": ns.N, "nnz": int(op["col"].numel()), "dt": dt, "steps": k * nsamp,
           "t_star": (np.arange(nsamp + 1) * sample).tolist(), "norm": norms.cpu().numpy().tolist(),
           "finite": bool(torch.isfinite(Q).all().item()), "build_s": build_s,
           "step_ms": ev0.elapsed_time(ev1) / (k * nsamp)}
    plan.close()
    return out


def _rates(runs, res):
    ref = np.array(runs[res[-1]]["norm"])
    err = {}
    for r in res[:-1]:
        d = np.array(runs[r]["norm"]) - ref
        err[r] = float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(ref * ref)))
    rates = {f"{a}-{b}": float(np.log(err[a] / err[b]) / np.log(b / a)) for a, b in zip(res[:-2], res[1:-1])}
    return err, rates


def study(lb, torch, resolutions=None, extra=(24,), **kw) -> dict:
    """All resolutions, the error of each against the finest printed one (R_c/s = 16)
    and the rates between consecutive resolutions (log of the error ratio over log of
    the resolution ratio: four rates for five coarser resolutions).  The paper prints
    five rates for those five without saying how the fifth is formed; with ``extra``
    finer runs, the same errors and rates against the finest of them as well (five
    rates, 3-4 to 12-16, when the extra run is R_c/s = 24)."""
    res = printed()[0] if resolutions is None else list(resolutions)
    allres = res + [r for r in extra if r not in res]
    runs = {r: run(lb, torch, r, **kw) for r in allres}
    err, rates = _rates(runs, res)
    out = {"runs": runs, "error_vs_finest": err, "rates": rates}
    if len(allres) > len(res):
        err2, rates2 = _rates(runs, allres)
        out[f"error_vs_{allres[-1]}"] = err2
        out[f"rates_vs_{allres[-1]}"] = rates2
    return out
