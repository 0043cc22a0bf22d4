"""Pins of the oracle's hand-derived adjoint: every vector-Jacobian product is
checked against central finite differences of the oracle's own forward map
(dot-product test <J v, m> = <v, J^T m>), so an error in the derivation (a
missing term, a wrong sign or coefficient) fails here."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as o

C2, MU = 100.0, 0.005


@pytest.fixture(scope="module")
def small():
    ns = li.tgv_lattice(14, 12, m=4, h_over_s=1.7, jitter=0.3, seed=31)
    rp, col = o.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    out = o.build_weights(ns.xy, ns.h, ns.s, rp, col, 4, ns.Lx, ns.Ly)
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=3)
    return ns, rp, col, out["w"], out["kappa"], q


def _fd(fun, q, v, eps):
    return (fun(q + eps * v) - fun(q - eps * v)) / (2 * eps)


def test_rhs_vjp_dot_product(small):
    ns, rp, col, w, kap, q = small
    rng = np.random.default_rng(0)
    for trial in range(3):
        v = rng.standard_normal(q.shape)
        m = rng.standard_normal(q.shape)
        jv = _fd(lambda x: o.rhs(x, w, rp, col, C2, MU), q, v, 1e-6)
        lhs = np.sum(jv * m)
        rhs_ = np.sum(v * o.rhs_vjp(q, m, w, rp, col, C2, MU))
        assert abs(lhs - rhs_) <= 1e-7 * abs(rhs_), (lhs, rhs_)


def test_rhs_vjp_each_field(small):
    # a perturbation of a single field and a cotangent on a single field at a time
    ns, rp, col, w, kap, q = small
    rng = np.random.default_rng(1)
    for fi in range(3):
        for fo in range(3):
            v = np.zeros_like(q)
            v[fi] = rng.standard_normal(q.shape[1])
            m = np.zeros_like(q)
            m[fo] = rng.standard_normal(q.shape[1])
            jv = _fd(lambda x: o.rhs(x, w, rp, col, C2, MU), q, v, 1e-6)
            lhs = np.sum(jv * m)
            rhs_ = np.sum(v * o.rhs_vjp(q, m, w, rp, col, C2, MU))
            assert abs(lhs - rhs_) <= 1e-7 * max(abs(rhs_), 1e-3 * np.abs(jv).max()), (fi, fo)


def test_filter_vjp_is_exact_transpose(small):
    ns, rp, col, w, kap, q = small
    rng = np.random.default_rng(2)
    v = rng.standard_normal(q.shape)
    m = rng.standard_normal(q.shape)
    lhs = np.sum(o.filter_fields(v, w[5], kap, rp, col) * m)
    rhs_ = np.sum(v * o.filter_vjp(m, w[5], kap, rp, col))
    assert abs(lhs - rhs_) <= 1e-12 * abs(rhs_)


def test_time_step_vjp_dot_product(small):
    ns, rp, col, w, kap, q = small
    dt = o.stable_dt(q, ns.s, 10.0, MU)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(q.shape)
    m = rng.standard_normal(q.shape)
    step = lambda x: o.time_step(x, dt, w, kap, rp, col, C2, MU)
    lhs = np.sum(_fd(step, q, v, 1e-6) * m)
    rhs_ = np.sum(v * o.time_step_vjp(q, m, dt, w, kap, rp, col, C2, MU))
    assert abs(lhs - rhs_) <= 1e-8 * abs(rhs_), (lhs, rhs_)


def test_rk_vjp_on_linear_ode_is_transpose_of_amplification():
    # for f(x) = A x the step is a matrix polynomial S(dt A); its VJP is S(dt A)^T
    rng = np.random.default_rng(4)
    A = rng.standard_normal((5, 5))
    f = lambda x: A @ x
    fv = lambda x, m: A.T @ m
    dt = 0.1
    S = np.stack([o.rk_step(e, dt, f) for e in np.eye(5)], axis=1)
    lam = rng.standard_normal(5)
    assert np.allclose(o.rk_step_vjp(np.zeros(5), lam, dt, f, fv), S.T @ lam, rtol=1e-13, atol=1e-13)


def test_conversions_and_energy_gradient(small):
    ns, rp, col, w, kap, q = small
    c = o.primitive_to_conserved(q)
    assert np.allclose(o.conserved_to_primitive(c), q, rtol=1e-14, atol=1e-15)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(c.shape)
    m = rng.standard_normal(c.shape)
    jv = _fd(o.conserved_to_primitive, c, v, 1e-7)
    assert np.isclose(np.sum(jv * m), np.sum(v * o.conserved_vjp(c, m)), rtol=1e-7)
    dq = rng.standard_normal(q.shape)
    ke = lambda x: o.kinetic_energy(x, ns.s)
    assert np.isclose((ke(q + 1e-6 * dq) - ke(q - 1e-6 * dq)) / 2e-6,
                      np.sum(dq * o.kinetic_energy_grad(q, ns.s)), rtol=1e-7)


def test_probe_momentum_and_gradient(small):
    ns, rp, col, w, kap, q = small
    rng = np.random.default_rng(7)
    # a smooth probe around (0.4, 0.6): closed form on a uniform state
    r2 = (ns.xy[:, 0] - 0.4) ** 2 + (ns.xy[:, 1] - 0.6) ** 2
    px, py = np.exp(-r2 / 0.02), 0.5 * np.exp(-r2 / 0.05)
    qu = np.stack([np.full(ns.N, np.log(1.2)), np.full(ns.N, 0.3), np.full(ns.N, -0.1)])
    assert o.probe_momentum(qu, px, py) == pytest.approx(1.2 * (0.3 * px.sum() - 0.1 * py.sum()),
                                                         rel=1e-14)
    g = o.probe_momentum_grad(q, px, py)
    for _ in range(3):
        v = rng.standard_normal(q.shape)
        fd = _fd(lambda x: o.probe_momentum(x, px, py), q, v, 1e-6)
        assert fd == pytest.approx(float(np.sum(g * v)), rel=1e-8)
