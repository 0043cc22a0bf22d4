"""Pins of the oracle's open boundaries (Section 7.1: outflow, eq. outflowL, and
inflow in LODI form) on a box bounded in x and periodic in y: uniform flow is an
exact steady state; on uniform states every derivative vanishes and the boundary
right-hand sides reduce to the closed forms of the relaxation terms, with the
printed coefficient from tests/golden; an acoustic pulse leaves through the
outflow with a small reflection, where a wall in its place reflects it fully."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import boundary_oracle as bo
from oracle import core as o
from tests.conftest import golden

C, U0, MU = 20.0, 1.0, 1e-3


def _sigma():
    return {k: float(v) for k, v in golden("nscbc.txt")}["sigma"]


@pytest.fixture(scope="module")
def box():
    ns = li.open_box(40, 12, m=6, jitter=0.05, seed=1)
    op = bo.channel_operator(ns, 6, 4)
    cols, normals = li.channel_walls(ns)
    n_b = cols.shape[0] // 2
    kind = np.array([bo.INFLOW] * n_b + [bo.OUTFLOW] * n_b)
    target = np.zeros((2 * n_b, 2))
    target[:n_b, 0] = U0        # inflow: u_xi,IN = U0 along the inward normal +x
    target[n_b:, 0] = C * C     # outflow: p_inf = c^2 rho0, rho0 = 1
    bnd = {"nodes": cols[:, 0], "normal": normals, "kind": kind, "target": target,
           "L": ns.Lx, "mach": U0 / C, "rho0": 1.0, "sigma": _sigma()}
    return ns, op, bnd


def _uniform(ns, a=0.0, u=U0, v=0.0):
    q = np.zeros((3, ns.N))
    q[0], q[1], q[2] = a, u, v
    return q


def test_uniform_flow_is_an_exact_steady_state(box):
    ns, op, bnd = box
    R = bo.boundary_rhs(_uniform(ns), op, bnd, C, MU)
    assert np.all(R == 0.0)


def test_outflow_relaxes_the_pressure_at_the_printed_rate(box):
    ns, op, bnd = box
    sigma, M, L = _sigma(), U0 / C, ns.Lx
    rho = 1.01
    R = bo.boundary_rhs(_uniform(ns, a=np.log(rho)), op, bnd, C, MU)
    out = bnd["nodes"][bnd["kind"] == bo.OUTFLOW]
    inn = bnd["nodes"][bnd["kind"] == bo.INFLOW]
    L4 = sigma / (2 * L) * C * (1 - M * M) * (C * C * rho - C * C)
    # d ln rho/dt = -L4 / (rho c^2); d u_xi/dt = -L4 / (rho c) with xi = -x at the outflow
    assert np.allclose(R[0, out], -L4 / (rho * C * C), rtol=1e-12, atol=0)
    assert np.allclose(R[1, out], +L4 / (rho * C), rtol=1e-12, atol=0)
    assert np.all(np.abs(R[2, out]) <= 1e-12)
    # the inflow sees its target velocity: nothing to relax
    assert np.all(np.abs(R[:, inn]) <= 1e-12)
    # the interior is uniform: eq. icns gives zero
    interior = np.setdiff1d(np.arange(ns.N), bnd["nodes"])
    assert np.all(R[:, interior] == 0.0)


def test_inflow_relaxes_both_velocity_components_at_the_printed_rates(box):
    ns, op, bnd = box
    sigma, M, L = _sigma(), U0 / C, ns.Lx
    du, dv = 0.01, -0.02
    R = bo.boundary_rhs(_uniform(ns, u=U0 + du, v=dv), op, bnd, C, MU)
    inn = bnd["nodes"][bnd["kind"] == bo.INFLOW]
    out = bnd["nodes"][bnd["kind"] == bo.OUTFLOW]
    L4 = sigma * 1.0 * C * C * (1 - M * M) / L * du   # rho0 = rho = 1, normal +x
    L3 = sigma * C / L * dv                            # tangent (0, 1): u_eta = v
    assert np.allclose(R[0, inn], -L4 / (C * C), rtol=1e-12, atol=0)
    assert np.allclose(R[1, inn], -L4 / C, rtol=1e-12, atol=0)
    assert np.allclose(R[2, inn], -L3, rtol=1e-12, atol=0)
    # the outflow sees p = p_inf and no gradients: nothing incoming to correct
    assert np.all(np.abs(R[:, out]) <= 1e-12)


def _pulse_run(kind_right):
    """A right-going acoustic pulse (u' = c a') in fluid at rest on the box with an
    inflow (target velocity zero) on the left and an outflow (or a wall) on the
    right, run until the pulse has reached the right boundary and a reflected pulse
    would be a quarter of the box back."""
    ns = li.open_box(96, 12, m=6, jitter=0.05, seed=2)
    op = bo.channel_operator(ns, 6, 4)
    cols, normals = li.channel_walls(ns)
    n_b = cols.shape[0] // 2
    kind = np.array([bo.INFLOW] * n_b + [kind_right] * n_b)
    target = np.zeros((2 * n_b, 2))
    target[n_b:, 0] = C * C
    bnd = {"nodes": cols[:, 0], "normal": normals, "kind": kind, "target": target,
           "L": ns.Lx, "mach": 0.0, "rho0": 1.0, "sigma": _sigma()}
    A, x0, w = 1e-3, 0.6 * ns.Lx, 0.3
    x = ns.xy[:, 0]
    pulse = A * np.exp(-((x - x0) / w) ** 2)
    q = _uniform(ns, u=0.0)
    q[0] += pulse
    q[1] += C * pulse
    dt = o.stable_dt(q, ns.s, C, MU)
    t_end = (ns.Lx - x0 + 0.25 * ns.Lx) / C
    for _ in range(int(np.ceil(t_end / dt))):
        q = bo.boundary_time_step(q, dt, op, bnd, C, MU)
    away = (x > 0.2 * ns.Lx) & (x < 0.85 * ns.Lx)
    return float(np.abs(q[0][away]).max()) / A, q


@pytest.mark.slow
def test_acoustic_pulse_leaves_through_the_outflow():
    out, q = _pulse_run(bo.OUTFLOW)
    wall, _ = _pulse_run(bo.WALL)
    assert np.all(np.isfinite(q))
    assert 0.8 < wall < 1.2, wall  # the wall sends the pulse back whole
    assert out < 0.05, out         # the outflow lets it through
