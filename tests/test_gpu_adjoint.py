"""The hand-written adjoint on the GPU against the FP64 oracle's adjoint and
against central finite differences of the GPU's own forward map."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, MU = 10.0, 0.005


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2102_02019_gb300 as lb
    return lb


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _case(lb, ns):
    rp, col = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    ow = oracle.build_weights(ns.xy, ns.h, ns.s, rp, col, ns.m, ns.Lx, ns.Ly)
    plans = {}
    for dt_ in (torch.float64, torch.float32):
        plan = lb.Plan(_dev(rp, torch.int32), _dev(col, torch.int32), _dev(ow["w"]), _dev(ow["kappa"]),
                       _dev(ns.s), dtype=dt_)
        lb.enable_adjoint(plan)
        plans[dt_] = plan
    return dict(ns=ns, rp=rp, col=col, w=ow["w"], kappa=ow["kappa"], plans=plans, s=_dev(ns.s))


@pytest.fixture(scope="module")
def stable(lb):
    # multi-step gradients need a trajectory that stays bounded: the raw +-0.3 s
    # jitter makes the locally tuned filter amplify a few modes (see the design
    # notes), so the rollouts use the +-0.1 s lattice
    return _case(lb, li.tgv_lattice(36, 32, m=4, h_over_s=1.7, jitter=0.1, seed=52))


@pytest.fixture(scope="module")
def case(lb):
    return _case(lb, li.tgv_lattice(40, 36, m=6, h_over_s=2.2, jitter=0.3, seed=51))


def test_rhs_adjoint_matches_oracle(lb, case):
    ns = case["ns"]
    q = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=4)
    m = np.random.default_rng(0).standard_normal(q.shape)
    phys = lb.Phys(C * C, MU)
    got = lb.rhs_adjoint(case["plans"][torch.float64], _dev(q), _dev(m), phys).cpu().numpy()
    ref = oracle.rhs_vjp(q, m, case["w"], case["rp"], case["col"], C * C, MU)
    assert np.all(_rel(got, ref) <= 1e-12), _rel(got, ref)


def test_filter_adjoint_matches_oracle(lb, case):
    ns = case["ns"]
    m = np.random.default_rng(1).standard_normal((3, ns.N))
    got = lb.filter_adjoint(case["plans"][torch.float64], _dev(m)).cpu().numpy()
    ref = oracle.filter_vjp(m, case["w"][5], case["kappa"], case["rp"], case["col"])
    assert np.all(_rel(got - m, ref - m) <= 1e-12)


def test_rk_step_adjoint_matches_oracle(lb, case):
    ns = case["ns"]
    q = li.tgv_fields(ns.xy, C)
    dt = oracle.stable_dt(q, ns.s, C, MU)
    m = np.random.default_rng(2).standard_normal(q.shape)
    lam = _dev(m)
    lb.rk_step_adjoint(case["plans"][torch.float64], _dev(q), lam, dt, lb.Phys(C * C, MU))
    ref = oracle.time_step_vjp(q, m, dt, case["w"], case["kappa"], case["rp"], case["col"], C * C, MU)
    got = lam.cpu().numpy()
    assert np.all(_rel(got, ref) <= 1e-12), _rel(got, ref)


def _ke_gradient(lb, plan, c0, s, dt, nsteps, every):
    c = c0.clone().requires_grad_(True)
    q = lb.to_primitive(c)
    qf = lb.rollout(plan, q, dt, nsteps, lb.Phys(C * C, MU), checkpoint_every=every)
    ke = lb.domain_kinetic_energy(qf, s)
    ke.backward()
    return float(ke.item()), c.grad.detach()


def test_kinetic_energy_gradient_matches_oracle_chain(lb, stable):
    case = stable
    ns = case["ns"]
    q0 = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=8)
    c0 = oracle.primitive_to_conserved(q0)
    dt = oracle.stable_dt(q0, ns.s, C, MU)
    nsteps, every = 7, 3
    ke, grad = _ke_gradient(lb, case["plans"][torch.float64], _dev(c0), case["s"], dt, nsteps, every)
    # oracle: forward storing states, reverse with the step VJP
    w, kap, rp, col = case["w"], case["kappa"], case["rp"], case["col"]
    states = [q0]
    for _ in range(nsteps):
        states.append(oracle.time_step(states[-1], dt, w, kap, rp, col, C * C, MU))
    assert abs(ke - oracle.kinetic_energy(states[-1], ns.s)) <= 1e-12 * ke
    lam = oracle.kinetic_energy_grad(states[-1], ns.s)
    for k in range(nsteps - 1, -1, -1):
        lam = oracle.time_step_vjp(states[k], lam, dt, w, kap, rp, col, C * C, MU)
    ref = oracle.conserved_vjp(c0, lam)
    got = grad.cpu().numpy()
    assert np.all(_rel(got, ref) <= 1e-10), _rel(got, ref)


def test_kinetic_energy_gradient_matches_central_differences(lb, stable):
    case = stable
    ns = case["ns"]
    plan = case["plans"][torch.float64]
    q0 = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=8)
    c0 = _dev(oracle.primitive_to_conserved(q0))
    dt = oracle.stable_dt(q0, ns.s, C, MU)
    nsteps = 6
    _, grad = _ke_gradient(lb, plan, c0, case["s"], dt, nsteps, 4)
    phys = lb.Phys(C * C, MU)

    def J(c):
        q = lb.conserved_to_primitive(c)
        lb.rk_step(plan, q, dt, nsteps, phys)
        return float(lb.kinetic_energy(q, case["s"]).item())

    rng = np.random.default_rng(3)
    eps = 1e-6
    for _ in range(3):
        v = _dev(rng.standard_normal((3, ns.N)))
        fd = (J(c0 + eps * v) - J(c0 - eps * v)) / (2 * eps)
        ad = float((grad * v).sum().item())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_fp32_rhs_adjoint_within_budget(lb, case):
    # the FP32 right-hand-side adjoint against the oracle's FP64 one, elementwise,
    # within the budget derived in tests/fp32_budget.py
    from tests.fp32_budget import rhs_vjp_bound
    ns = case["ns"]
    q = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=4)
    m = np.random.default_rng(4).standard_normal(q.shape)
    got = lb.rhs_adjoint(case["plans"][torch.float32], _dev(q, torch.float32), _dev(m, torch.float32),
                         lb.Phys(C * C, MU)).double().cpu().numpy()
    ref = oracle.rhs_vjp(q, m, case["w"], case["rp"], case["col"], C * C, MU)
    bound = rhs_vjp_bound(q, m, case["w"], case["rp"], case["col"], C * C, MU,
                          G=case["plans"][torch.float32].info()["group"])
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, ratio.max()
    print("FP32 RHS adjoint: max error / budget", ratio.max(), "rel L2", _rel(got, ref))


def test_fp32_filter_adjoint_within_budget(lb, case):
    from tests.fp32_budget import filter_vjp_bound
    ns = case["ns"]
    lam = np.random.default_rng(5).standard_normal((3, ns.N))
    got = lb.filter_adjoint(case["plans"][torch.float32], _dev(lam, torch.float32)).double().cpu().numpy()
    ref = oracle.filter_vjp(lam, case["w"][5], case["kappa"], case["rp"], case["col"])
    bound = filter_vjp_bound(lam, ref, case["w"][5], case["kappa"], case["rp"], case["col"],
                             G=case["plans"][torch.float32].info()["group"])
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, ratio.max()


def test_fp32_step_adjoint_within_budget(lb, case):
    # one reverse time step in FP32 against the oracle's FP64 transpose of the step
    from tests.fp32_budget import step_vjp_bound
    ns = case["ns"]
    q = li.tgv_fields(ns.xy, C)
    dt = oracle.stable_dt(q, ns.s, C, MU)
    m = np.random.default_rng(4).standard_normal(q.shape)
    lam = _dev(m, torch.float32)
    lb.rk_step_adjoint(case["plans"][torch.float32], _dev(q, torch.float32), lam, dt, lb.Phys(C * C, MU))
    got = lam.double().cpu().numpy()
    ref = oracle.time_step_vjp(q, m, dt, case["w"], case["kappa"], case["rp"], case["col"], C * C, MU)
    bound = step_vjp_bound(q, m, ref, dt, case["w"], case["kappa"], case["rp"], case["col"], C * C, MU,
                           G=case["plans"][torch.float32].info()["group"])
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, ratio.max()
    print("FP32 step adjoint: max error / budget", ratio.max(), "rel L2", _rel(got, ref))


def _probe(ns):
    r2 = (ns.xy[:, 0] - 0.4) ** 2 + (ns.xy[:, 1] - 0.6) ** 2
    return np.exp(-r2 / 0.02), 0.5 * np.exp(-r2 / 0.05)


def test_probe_momentum_matches_oracle(lb, case):
    ns = case["ns"]
    px, py = _probe(ns)
    q = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=4)
    j = float(lb.probe_momentum(_dev(q), _dev(px), _dev(py)).item())
    assert j == pytest.approx(oracle.probe_momentum(q, px, py), rel=1e-13)
    g = lb.probe_momentum_grad(_dev(q), _dev(px), _dev(py), 2.0).cpu().numpy()
    assert np.all(_rel(g, 2.0 * oracle.probe_momentum_grad(q, px, py)) <= 1e-14)


def test_probe_momentum_gradient_through_rollout(lb, stable):
    # gradient of the final probe-weighted momentum w.r.t. the initial conserved
    # state: the oracle's adjoint chain and central differences of the GPU forward
    case = stable
    ns = case["ns"]
    px, py = _probe(ns)
    q0 = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=8)
    c0 = oracle.primitive_to_conserved(q0)
    dt = oracle.stable_dt(q0, ns.s, C, MU)
    nsteps = 5
    plan = case["plans"][torch.float64]
    phys = lb.Phys(C * C, MU)
    pxd, pyd = _dev(px), _dev(py)
    c = _dev(c0).requires_grad_(True)
    qf = lb.rollout(plan, lb.to_primitive(c), dt, nsteps, phys, checkpoint_every=2)
    J = lb.domain_probe_momentum(qf, pxd, pyd)
    J.backward()
    grad = c.grad.detach()
    w, kap, rp, col = case["w"], case["kappa"], case["rp"], case["col"]
    states = [q0]
    for _ in range(nsteps):
        states.append(oracle.time_step(states[-1], dt, w, kap, rp, col, C * C, MU))
    assert float(J.item()) == pytest.approx(oracle.probe_momentum(states[-1], px, py), rel=1e-12)
    lam = oracle.probe_momentum_grad(states[-1], px, py)
    for k in range(nsteps - 1, -1, -1):
        lam = oracle.time_step_vjp(states[k], lam, dt, w, kap, rp, col, C * C, MU)
    ref = oracle.conserved_vjp(c0, lam)
    assert np.all(_rel(grad.cpu().numpy(), ref) <= 1e-10)

    def Jf(cc):
        q = lb.conserved_to_primitive(cc)
        lb.rk_step(plan, q, dt, nsteps, phys)
        return float(lb.probe_momentum(q, pxd, pyd).item())

    v = _dev(np.random.default_rng(8).standard_normal((3, ns.N)))
    fd = (Jf(_dev(c0) + 1e-6 * v) - Jf(_dev(c0) - 1e-6 * v)) / 2e-6
    ad = float((grad * v).sum().item())
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_recorded_step_and_adjoint_equal_the_recomputing_ones(lb, case, dtype):
    ns = case["ns"]
    plan = case["plans"][dtype]
    q = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=4)
    dt = oracle.stable_dt(q, ns.s, C, MU)
    phys = lb.Phys(C * C, MU)
    m = np.random.default_rng(9).standard_normal(q.shape)
    Qa, Qb = _dev(q, dtype), _dev(q, dtype)
    X = lb.stage_states(plan)
    lb.rk_step_record(plan, Qa, X, dt, phys)
    lb.rk_step(plan, Qb, dt, 1, phys)
    assert torch.equal(Qa, Qb)
    la, lbb = _dev(m, dtype), _dev(m, dtype)
    lb.rk_step_adjoint_recorded(plan, X, la, dt, phys)
    lb.rk_step_adjoint(plan, _dev(q, dtype), lbb, dt, phys)
    assert torch.equal(la, lbb)
