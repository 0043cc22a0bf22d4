"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws node sets and initial fields.  It holds none of the
LABFM arithmetic (no basis functions, no weights, no derivative operators):
both the CPU oracle and the CUDA path consume what it returns.

Workloads (all doubly periodic, unit square unless stated):

* ``tgv_lattice(nx, ...)``: the jittered Cartesian node set of the paper's
  uniform-resolution tests (Section 5: a lattice with spacing s, every node
  shifted by a random vector), node ``(ix, iy)`` at
  ``((ix + 0.5 + U[-j, j]) s, (iy + 0.5 + U[-j, j]) s)`` with ``j = 0.3``,
  optionally followed by iterations of the paper's iterative shifting
  (``shift_iterations``, see ``iterative_shift``).  Nodes are numbered row by
  row (x fastest).
* ``varres_columns(s0, ...)``: variable resolution ``s(x) = s0 (1 + 1.5 sin^2(pi x))``
  built from periodic columns; each node's stencil scale gets a seeded
  multiplier (the spread that stencil optimisation leaves, Section 4).
* ``batch_instances(...)``: many independent lattices with log-uniform sizes and
  mixed orders m in {4, 6, 8}.
* ``tgv_fields(xy, c)``: the Taylor-Green initial condition of Section 8.1 in the
  evolved variables (ln rho, u, v), with rho = 1 + p / c^2.
* ``channel(nx, ny, ...)``: a channel periodic in x between two walls, with the five
  uniform node rows along each wall that the boundary scheme of Section 7.1 needs;
  ``channel_walls(ns)`` lists its wall nodes' normal columns and normals.
* ``open_box(nx, ny, ...)``: the same layout turned by 90 degrees, bounded in x by an
  inflow (x = 0) and an outflow (x = Lx), periodic in y (Section 8.3's domain).
* ``lamb_oseen_fields(xy, c, ...)``: Section 8.3's Lamb-Oseen vortex on a uniform
  stream in (ln rho, u, v), centred in the unit box.
* ``smooth_perturbation(xy, ...)``: a seeded band-limited random field
  (integer wavevectors with |k| <= kmax), normalised to unit maximum amplitude.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2102_02019

# h/s used for each order when a workload mixes orders (m=4 and m=8 follow the
# two lattice workloads; m=6 uses the "safe" non-optimised value of Section 4).
H_OVER_S = {2: 1.2, 4: 1.7, 6: 2.2, 8: 2.8, 10: 3.3}


@dataclass
class NodeSet:
    """A node distribution: positions, spacing s_i and stencil scale h_i."""

    xy: np.ndarray  # (N, 2) float64, inside [0, Lx) x [0, Ly)
    s: np.ndarray  # (N,) float64
    h: np.ndarray  # (N,) float64
    Lx: float
    Ly: float
    m: int
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.xy.shape[0])


def rng_for(config_index: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for a workload; ``stream`` separates independent draws."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + config_index, stream]))


# Support of the iterative shifting in units of s.  The paper gives none.  A scan
# of supports from 2 s to 5 s (0.5 s steps; 5, 10 and 20 iterations) on 40 x 40
# lattices jittered by +-0.3 s found 3.5 s to be the only one whose shifted node
# sets give time steps that stay finite for m = 4, 6 and 8 (largest filter
# coefficient 2.3-3.5 times the median, against 4-80 times otherwise); ten
# iterations leave every node 0.13 s (rms; at most 0.34 s) from its lattice site
# and no two nodes closer than 0.85 s.
SHIFT_H_OVER_S = 3.5
# Iterations the paper applies to its uniform-resolution node sets (Section 5).
SHIFT_ITERATIONS = 10


def iterative_shift(xy: np.ndarray, s: np.ndarray, Lx: float, Ly: float, iterations: int,
                    h_over_s: float = SHIFT_H_OVER_S) -> np.ndarray:
    """Iterative shifting of a periodic node set (Section 5, eq. iter_shift):

        r_i <- r_i + (s_i^2 / h_i) sum_{j : |r_ji| < h_i} (|r_ji| / h_i - 1) r_ji / |r_ji|

    with r_ji = r_j - r_i on the periodic minimum image, all nodes moved at once
    (Jacobi) in each iteration, and positions wrapped back into the box.  The
    paper writes one h without a value; here h_i = h_over_s s_i.  Every term
    pushes node i away from a neighbour closer than h_i, so close pairs separate
    and the spacing evens out.  This is node generation, not LABFM arithmetic."""
    from scipy.spatial import cKDTree

    pos = np.array(xy, dtype=np.float64)
    N = pos.shape[0]
    box = np.array([Lx, Ly])
    h = h_over_s * np.asarray(s, dtype=np.float64)
    hmax = float(np.max(h))
    for _ in range(iterations):
        pos = np.mod(pos, box)
        pos[pos >= box] = 0.0  # mod can round up to the box size
        tree = cKDTree(pos, boxsize=box)
        pairs = tree.query_pairs(hmax, output_type="ndarray")
        i, j = pairs[:, 0], pairs[:, 1]
        d = pos[j] - pos[i]
        d -= box * np.round(d / box)  # minimum image
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        keep = r > 0.0
        i, j, d, r = i[keep], j[keep], d[keep], r[keep]
        unit = d / r[:, None]
        shift = np.zeros_like(pos)
        # each pair contributes to both ends, each with its own h (r_ij = -r_ji)
        for a, sign in ((i, 1.0), (j, -1.0)):
            ha = h[a]
            inside = r < ha
            coef = sign * (s[a] ** 2 / ha) * (r / ha - 1.0) * inside
            shift[:, 0] += np.bincount(a, weights=coef * unit[:, 0], minlength=N)
            shift[:, 1] += np.bincount(a, weights=coef * unit[:, 1], minlength=N)
        pos = pos + shift
    pos = np.mod(pos, box)
    pos[pos >= box] = 0.0
    return pos


def tgv_lattice(nx: int, ny: int | None = None, m: int = 4, h_over_s: float | None = None,
                jitter: float = 0.3, seed: int = 0, s: float | None = None,
                shift_iterations: int = 0) -> NodeSet:
    """Jittered nx x ny lattice with spacing s (default 1/nx) on [0, nx s) x [0, ny s),
    then `shift_iterations` iterations of iterative shifting (Section 5; the paper
    applies 10 to its uniform-resolution node sets)."""
    ny = nx if ny is None else ny
    s = 1.0 / nx if s is None else s
    if h_over_s is None:
        h_over_s = H_OVER_S[m]
    rng = rng_for(seed, 0)
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    jx = rng.uniform(-jitter, jitter, size=(ny, nx))
    jy = rng.uniform(-jitter, jitter, size=(ny, nx))
    x = (ix + 0.5 + jx) * s
    y = (iy + 0.5 + jy) * s
    xy = np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float64)
    N = nx * ny
    sv = np.full(N, s, dtype=np.float64)
    hv = np.full(N, h_over_s * s, dtype=np.float64)
    if shift_iterations:
        xy = iterative_shift(xy, sv, nx * s, ny * s, shift_iterations)
    return NodeSet(xy, sv, hv, nx * s, ny * s, m,
                   {"kind": "lattice", "nx": nx, "ny": ny, "jitter": jitter, "seed": seed,
                    "h_over_s": h_over_s, "shift_iterations": shift_iterations})


def varres_spacing(x: np.ndarray, s0: float) -> np.ndarray:
    """s(x) = s0 (1 + 1.5 sin^2(pi x)) for the variable-resolution box."""
    return s0 * (1.0 + 1.5 * np.sin(np.pi * x) ** 2)


def varres_columns(s0: float = 6.654e-4, m: int = 10, h_over_s: float = 3.3,
                   h_spread=(0.85, 1.25), jitter: float = 0.3, seed: int = 2,
                   h_field: str = "random", shift_iterations: int = 0) -> NodeSet:
    """Periodic columns whose spacing follows s(x) = s0 (1 + 1.5 sin^2 pi x).

    Column positions advance by s(x_k) and are rescaled to close at x = 1;
    column k holds round(1/s(x_k)) evenly spaced nodes in y.  Every node is
    jittered by +-0.3 s in both directions and gets h_i = h_over_s * s_i * M_i
    with M_i in h_spread: independent uniform draws (``h_field="random"``) or a
    smooth field, the midpoint of h_spread plus its half-width times a seeded
    band-limited field of unit maximum amplitude (wavevectors |k| <= 2;
    ``h_field="smooth"``), so that neighbouring stencils have nearly the same
    size.  ``shift_iterations`` iterations of iterative shifting (Section 5) move
    the nodes after the jitter (each keeps its column's s).
    """
    xs = [0.0]
    while True:
        nxt = xs[-1] + float(varres_spacing(np.array([xs[-1]]), s0)[0])
        if nxt >= 1.0:
            break
        xs.append(nxt)
    xs = np.asarray(xs)
    xs = xs * (1.0 / (xs[-1] + varres_spacing(np.array([xs[-1]]), s0)[0]))
    # centre each column in its own slab
    widths = np.diff(np.append(xs, 1.0))
    xc = xs + 0.5 * widths
    rng = rng_for(seed, 0)
    rows_x, rows_y, rows_s = [], [], []
    for k in range(len(xc)):
        sk = float(varres_spacing(np.array([xc[k]]), s0)[0])
        ny = max(1, int(round(1.0 / sk)))
        sy = 1.0 / ny
        iy = np.arange(ny)
        y = (iy + 0.5 + rng.uniform(-jitter, jitter, size=ny)) * sy
        x = xc[k] + rng.uniform(-jitter, jitter, size=ny) * widths[k]
        rows_x.append(np.mod(x, 1.0))
        rows_y.append(np.mod(y, 1.0))
        rows_s.append(np.full(ny, sk))
    x = np.concatenate(rows_x)
    y = np.concatenate(rows_y)
    s = np.concatenate(rows_s)
    xy = np.stack([x, y], axis=1)
    if shift_iterations:
        xy = iterative_shift(xy, s, 1.0, 1.0, shift_iterations)
    if h_field == "random":
        mult = rng_for(seed, 1).uniform(h_spread[0], h_spread[1], size=x.shape[0])
    elif h_field == "smooth":
        mid, half = 0.5 * (h_spread[0] + h_spread[1]), 0.5 * (h_spread[1] - h_spread[0])
        mult = mid + half * smooth_perturbation(xy, kmax=2, seed=seed + 100)
    else:
        raise ValueError("h_field must be 'random' or 'smooth'")
    h = h_over_s * s * mult
    return NodeSet(xy, s, h, 1.0, 1.0, m,
                   {"kind": "varres", "s0": s0, "columns": int(len(xc)), "seed": seed,
                    "h_over_s": h_over_s, "h_spread": list(h_spread), "h_field": h_field,
                    "shift_iterations": shift_iterations, "s_ratio": float(s.max() / s.min())})


def batch_instances(count: int = 256, n_min: int = 2048, n_max: int = 65536,
                    orders=(4, 6, 8), seed: int = 3) -> list[NodeSet]:
    """Independent jittered lattices, N log-uniform in [n_min, n_max], m uniform in orders."""
    rng = rng_for(seed, 0)
    logs = rng.uniform(math.log(n_min), math.log(n_max), size=count)
    ms = rng.choice(np.asarray(orders), size=count)
    out = []
    for k in range(count):
        nx = max(8, int(round(math.sqrt(math.exp(logs[k])))))
        m = int(ms[k])
        out.append(tgv_lattice(nx, nx, m=m, seed=1000 + 7 * k + seed))
    return out


def channel(nx: int, ny: int, m: int = 4, h_over_s: float | None = None, jitter: float = 0.3,
            seed: int = 0, h_wall_over_s: float = 2.2) -> NodeSet:
    """A channel periodic in x on [0, nx s) with walls at y = 0 and y = ny s (s = 1/nx):
    the node layout of Section 7.1 near walls.  Along each wall five uniform rows
    (row index q = 0 on the wall, q = 1..4 at q s along the inward normal) share
    their x positions ((ix + 0.5) s), so every wall node has its four normal
    neighbours; the rows in between are jittered lattice rows at y = iy s,
    iy = 5 .. ny - 5 (ny >= 10).  meta: ``row`` (q, or 5 in the interior),
    ``normal`` (inward unit normal of the nearest wall, zero in the interior),
    ``column`` (the node's x index in the uniform rows, -1 in the interior) and
    ``wall`` (0 bottom, 1 top, -1 interior).  The rows q = 1, 2, whose second
    derivatives come from one-sided order-4 stencils, get h = h_wall_over_s s (the
    paper gives no value; 2.2 s, its "safe" m = 6 scale, keeps those systems
    conditioned), every other node h = h_over_s s."""
    if ny < 10:
        raise ValueError("need ny >= 10: five uniform rows at each wall and a jittered interior")
    s = 1.0 / nx
    H = ny * s
    rng = rng_for(20, seed)
    xs, ys, row, nrm, colx, wall = [], [], [], [], [], []
    for w, (y0, sign) in enumerate(((0.0, 1.0), (H, -1.0))):
        for q in range(5):
            for ix in range(nx):
                xs.append((ix + 0.5) * s)
                ys.append(y0 + sign * q * s)
                row.append(q)
                nrm.append((0.0, sign))
                colx.append(ix)
                wall.append(w)
    for iy in range(5, ny - 4):
        for ix in range(nx):
            dx, dy = rng.uniform(-jitter, jitter, size=2)
            xs.append(((ix + 0.5 + dx) * s) % 1.0)
            ys.append((iy + dy) * s)
            row.append(5)
            nrm.append((0.0, 0.0))
            colx.append(-1)
            wall.append(-1)
    xy = np.stack([np.array(xs), np.array(ys)], axis=1)
    hs = H_OVER_S[m] if h_over_s is None else h_over_s
    N = xy.shape[0]
    rows = np.array(row)
    hv = np.where((rows == 1) | (rows == 2), h_wall_over_s * s, hs * s)
    return NodeSet(xy=xy, s=np.full(N, s), h=hv, Lx=1.0, Ly=H, m=m,
                   meta={"row": np.array(row), "normal": np.array(nrm), "column": np.array(colx),
                         "wall": np.array(wall), "nx": nx, "ny": ny, "h_over_s": hs})


def open_box(nx: int, ny: int, m: int = 6, h_over_s: float | None = None, jitter: float = 0.1,
             seed: int = 0, h_wall_over_s: float = 2.2) -> NodeSet:
    """A box bounded in x with open boundaries at x = 0 (inflow) and x = nx s
    (outflow), periodic in y on [0, ny s) (s = 1/ny): the ``channel`` node set with x
    and y exchanged, so that five uniform columns of nodes (q = 0 on the boundary,
    q = 1..4 at q s along the inward normal, the x axis) line each boundary and the
    nodes in between are a jittered lattice.  meta as for ``channel``; ``wall`` is 0
    for the boundary at x = 0 and 1 for x = nx s."""
    ch = channel(ny, nx, m=m, h_over_s=h_over_s, jitter=jitter, seed=seed, h_wall_over_s=h_wall_over_s)
    meta = dict(ch.meta)
    meta["normal"] = ch.meta["normal"][:, ::-1].copy()
    meta["nx"], meta["ny"] = nx, ny
    meta["kind"] = "open_box"
    return NodeSet(xy=ch.xy[:, ::-1].copy(), s=ch.s, h=ch.h, Lx=ch.Ly, Ly=ch.Lx, m=m, meta=meta)


def channel_walls(ns: NodeSet) -> tuple[np.ndarray, np.ndarray]:
    """The walls of a ``channel`` node set as Section 7.1 describes them: for every
    wall node b (row q = 0) its normal column, the nodes of rows q = 0..4 with the
    same wall and x index ((n_wall, 5) int32), and its inward unit normal
    ((n_wall, 2) float64).  Wall nodes are listed bottom wall first, by x index."""
    meta = ns.meta
    key = {(int(w), int(c), int(q)): k for k, (w, c, q) in
           enumerate(zip(meta["wall"], meta["column"], meta["row"])) if q < 5}
    cols, normals = [], []
    per_row = meta["ny"] if meta.get("kind") == "open_box" else meta["nx"]
    for w in (0, 1):
        for c in range(per_row):
            cols.append([key[(w, c, q)] for q in range(5)])
            normals.append(meta["normal"][key[(w, c, 0)]])
    return np.asarray(cols, dtype=np.int32), np.asarray(normals, dtype=np.float64)


def tgv_fields(xy: np.ndarray, c: float = 10.0, H: float = 1.0) -> np.ndarray:
    """Taylor-Green initial state (ln rho, u, v) as a (3, N) float64 array.

    u = -cos(2 pi x/H) sin(2 pi y/H), v = sin(2 pi x/H) cos(2 pi y/H),
    p = -(H/4)(cos(4 pi x/H) + cos(4 pi y/H)) and rho = 1 + p / c^2.
    """
    x = xy[:, 0]
    y = xy[:, 1]
    k = 2.0 * math.pi / H
    u = -np.cos(k * x) * np.sin(k * y)
    v = np.sin(k * x) * np.cos(k * y)
    p = -(H / 4.0) * (np.cos(2 * k * x) + np.cos(2 * k * y))
    rho = 1.0 + p / (c * c)
    return np.stack([np.log(rho), u, v]).astype(np.float64)


LAMB_OSEEN_RC_OVER_H = 1.0 / 25.0     # vortex radius R_c = H / 25 (Section 8.3)
LAMB_OSEEN_C_OVER_CH = 1.0 / 300.0    # vortex strength C = c H / 300
LAMB_OSEEN_RE = 7500.0                # Re = U0 R_c rho0 / mu
LAMB_OSEEN_MACH = 0.05                # Ma = U0 / c


def lamb_oseen_fields(xy: np.ndarray, c: float, U0: float = 1.0, H: float = 1.0, rho0: float = 1.0,
                      centre=(0.5, 0.5)) -> np.ndarray:
    """Section 8.3's initial state as (ln rho, u, v): a Lamb-Oseen vortex of radius R_c
    and strength C at ``centre`` on the uniform stream (U0, 0),
        (u, v) = (U0, 0) + (C/rho0) (y', -x') / R_c^2 exp(-r'^2 / (2 R_c^2)),
        rho = rho0 (1 - C^2 / (c^2 R_c^2) exp(-r'^2 / (2 R_c^2))),
    with (x', y') = (x, y) - centre and R_c, C from the printed ratios."""
    Rc = LAMB_OSEEN_RC_OVER_H * H
    C = LAMB_OSEEN_C_OVER_CH * c * H
    x = xy[:, 0] - centre[0]
    y = xy[:, 1] - centre[1]
    g = np.exp(-(x * x + y * y) / (2.0 * Rc * Rc))
    u = U0 + C / rho0 * y / (Rc * Rc) * g
    v = -C / rho0 * x / (Rc * Rc) * g
    rho = rho0 * (1.0 - C * C / (c * c * Rc * Rc) * g)
    return np.stack([np.log(rho), u, v]).astype(np.float64)


def smooth_perturbation(xy: np.ndarray, kmax: int = 8, seed: int = 4, stream: int = 0,
                        Lx: float = 1.0, Ly: float = 1.0) -> np.ndarray:
    """Sum over integer wavevectors 0 < |k| <= kmax of N(0,1) * cos / sin(2 pi k.x),
    normalised so that its maximum magnitude over the nodes is 1."""
    rng = rng_for(seed, 10 + stream)
    x = xy[:, 0] / Lx
    y = xy[:, 1] / Ly
    f = np.zeros(xy.shape[0])
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if (kx == 0 and ky == 0) or kx * kx + ky * ky > kmax * kmax:
                continue
            a, b = rng.standard_normal(2)
            ph = 2.0 * math.pi * (kx * x + ky * y)
            f += a * np.cos(ph) + b * np.sin(ph)
    return f / np.abs(f).max()


def perturbed_tgv_fields(xy: np.ndarray, c: float = 10.0, amplitude: float = 0.05,
                         kmax: int = 8, seed: int = 4) -> np.ndarray:
    """Taylor-Green state plus ``amplitude`` times an independent smooth field per variable."""
    q = tgv_fields(xy, c)
    for f in range(3):
        q[f] += amplitude * smooth_perturbation(xy, kmax=kmax, seed=seed, stream=f)
    return q


# Named workloads used by tests and the benchmark.
WORKLOADS = {
    "tgv64_m4": dict(nx=64, m=4, steps=100, c=10.0),
    "tgv512_m8": dict(nx=512, m=8, steps=1000, c=10.0),
}


def workload(name: str) -> NodeSet:
    cfg = WORKLOADS[name]
    idx = list(WORKLOADS).index(name)
    return tgv_lattice(cfg["nx"], m=cfg["m"], seed=idx)
