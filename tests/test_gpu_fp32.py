"""FP32 path (fields and nondimensionalised weights in float) against the FP64 oracle.

Budget, derived from the arithmetic (tests/fp32_budget.py).  With u = 2^-24 (float unit roundoff),
each input phi_j, each stored weight w~_ji and the scale 1/s_i carry a relative
rounding of u; phi_j - phi_i, the product and the compensated sum add a few
more.  For one derivative the error is therefore bounded by

    B_d,i = 3 u sum_j |w_ji| (|phi_j| + |phi_i|) + 2 u |L_d,i|

(the factor 3 covers weight, input and product roundings; the compensated sums
keep the summation error at O(u)).  The pointwise right-hand side propagates
these bounds linearly with absolute values and adds 4 u times the sum of the
absolute values of its terms.  Tests require |R32 - R64| <= B elementwise.
"""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.fp32_budget import U32, deriv_bound as _deriv_bound, rhs_bound, step_bound  # noqa: F401


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


@pytest.fixture(scope="module")
def setup(lb):
    ns = li.tgv_lattice(48, 40, m=8, h_over_s=2.8, jitter=0.3, seed=12)
    rp, col = oracle.neighbours(ns.xy, ns.h, ns.Lx, ns.Ly)
    ow = oracle.build_weights(ns.xy, ns.h, ns.s, rp, col, ns.m, ns.Lx, ns.Ly)
    rpd = _dev(rp, torch.int32)
    cold = _dev(col, torch.int32)
    plan32 = lb.Plan(rpd, cold, _dev(ow["w"]), _dev(ow["kappa"]), _dev(ns.s), dtype=torch.float32)
    return dict(ns=ns, rp=rp, col=col, ow=ow, plan32=plan32, s=_dev(ns.s))


def test_rhs_fp32_within_rounding_budget(lb, setup):
    ns, rp, col, ow = setup["ns"], setup["rp"], setup["col"], setup["ow"]
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.05, kmax=4)
    phys = lb.Phys(100.0, 0.005)
    R32 = lb.rhs(setup["plan32"], _dev(q, torch.float32), phys).double().cpu().numpy()
    R64 = oracle.rhs(q, ow["w"][:5], rp, col, 100.0, 0.005)
    B = rhs_bound(q, ow["w"], rp, col, 100.0, 0.005)
    ratio = np.abs(R32 - R64) / B
    assert ratio.max() <= 1.0, ratio.max()
    rel = np.linalg.norm(R32 - R64, axis=1) / np.linalg.norm(R64, axis=1)
    print("FP32 RHS rel L2 per field (ln rho, u, v):", rel, "max err/bound", ratio.max())


def test_filter_fp32_within_rounding_budget(lb, setup):
    ns, rp, col, ow = setup["ns"], setup["rp"], setup["col"], setup["ow"]
    q = li.perturbed_tgv_fields(ns.xy, 10.0, amplitude=0.1, kmax=8)
    F32 = lb.filter(setup["plan32"], _dev(q, torch.float32)).double().cpu().numpy()
    F64 = oracle.filter_fields(q, ow["w"][5], ow["kappa"], rp, col)
    wf = ow["w"][5] * np.repeat(ow["kappa"], np.diff(rp))
    for f in range(3):
        b, _ = _deriv_bound(q[f], wf, rp, col)
        bound = b + 2 * U32 * np.abs(q[f]) + 2 * U32 * np.abs(F64[f])
        assert np.all(np.abs(F32[f] - F64[f]) <= bound)


def test_rk_step_fp32_one_step(lb, setup):
    ns, rp, col, ow = setup["ns"], setup["rp"], setup["col"], setup["ow"]
    q0 = li.tgv_fields(ns.xy, 10.0)
    dt = oracle.stable_dt(q0, ns.s, 10.0, 0.005)
    Q = _dev(q0, torch.float32)
    lb.rk_step(setup["plan32"], Q, dt, 1, lb.Phys(100.0, 0.005))
    q1 = oracle.time_step(q0, dt, ow["w"], ow["kappa"], rp, col, 100.0, 0.005)
    # per node: storage rounding of Q, plus dt sum_k |b_k| times the RHS budget at the
    # initial state (the stage states differ from it by O(dt)), plus the filter budget
    bound = step_bound(q0, q1, dt, ow["w"], ow["kappa"], rp, col, 100.0, 0.005)
    got = Q.double().cpu().numpy()
    for f in range(3):
        assert np.all(np.abs(got[f] - q1[f]) <= bound[f]), (f, (np.abs(got[f] - q1[f]) / bound[f]).max())


def test_profiling_and_host_buffer_step(lb, setup):
    ns = setup["ns"]
    plan = setup["plan32"]
    q0 = li.tgv_fields(ns.xy, 10.0)
    Qd = _dev(q0, torch.float32)
    Qref = Qd.clone()
    work = lb.workspace(plan)
    plan.set_profiling(True)
    lb.rk_step(plan, Qref, 1e-4, 3, lb.Phys(100.0, 0.005), work=work)
    prof = plan.read_profile()
    plan.set_profiling(False)
    assert prof["stage_launches"] == 12 and prof["filter_launches"] == 3 and prof["dropped"] == 0
    assert prof["stage_ms"] > 0 and prof["filter_ms"] > 0
    # sampled: every 3rd of 7 steps (steps 0, 3, 6) carries the events
    plan.set_profiling(True, every=3)
    lb.rk_step(plan, Qref.clone(), 1e-4, 7, lb.Phys(100.0, 0.005), work=work)
    prof = plan.read_profile()
    plan.set_profiling(False)
    assert prof["stage_launches"] == 12 and prof["filter_launches"] == 3 and prof["dropped"] == 0
    with pytest.raises(lb.LabfmError):
        plan.set_profiling(True, every=-1)
    # pinned host memory (stepped in place over the host link) and pageable host
    # memory (staged through the device scratch) give the device result
    scratch = torch.empty_like(Qd)
    for Qh in (torch.tensor(q0, dtype=torch.float32).pin_memory(), torch.tensor(q0, dtype=torch.float32)):
        lb.rk_step_host(plan, Qh, scratch, 1e-4, 3, lb.Phys(100.0, 0.005), work=work)
        assert torch.equal(Qh, Qref.cpu())
