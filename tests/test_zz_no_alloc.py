"""labfm_rk_step_noalloc, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: a host application or plugin that gives the
library only memory it manages itself, or a real-time loop that must not pay for
or synchronise on an allocation.  For them labfm_rk_step_noalloc runs the same
RK step with its scratch in the library's static device array.  Its result must
match labfm_rk_step (which takes a caller-allocated work buffer) within the
tolerance of the other FP64 parity tests, on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next result).

This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2102_02019_gb300 as lb
    return lb


def _rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _noalloc_call(lb, plan, Q, dt, nsteps, phys):
    ph = phys.c()
    return lb.lib.labfm_rk_step_noalloc(plan.handle, Q.data_ptr(), float(dt), nsteps, ctypes.byref(ph),
                                        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype,tol,persistent", [(torch.float64, 1e-12, False), (torch.float32, 1e-6, False),
                                                  (torch.float32, 1e-6, True)])
def test_noalloc_step_matches_rk_step_twice(lb, dtype, tol, persistent):
    ns = li.tgv_lattice(48, 40, m=6, h_over_s=2.2, jitter=0.1, seed=13)
    dev = "cuda"
    xy = torch.tensor(ns.xy, device=dev)
    h = torch.tensor(ns.h, device=dev)
    s = torch.tensor(ns.s, device=dev)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, ns.m)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
    if persistent:
        # the work-queue tickets of a persistent plan live in the static array too
        plan.set_persistent(True)
    phys = lb.Phys(100.0, 0.005)
    q0 = li.tgv_fields(ns.xy, 10.0)
    dt = oracle.stable_dt(q0, ns.s, 10.0, 0.005)
    for call, (q_start, nsteps) in enumerate([(q0, 3), (li.perturbed_tgv_fields(ns.xy, 10.0), 2)]):
        Qa = torch.tensor(q_start, dtype=dtype, device=dev)
        Qb = Qa.clone()
        lb.rk_step(plan, Qa, dt, nsteps, phys)
        torch.cuda.synchronize()
        # through the C ABI directly: no work buffer, and nothing allocated by the
        # call (device memory as the CUDA driver and torch's allocator see it is unchanged)
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        rc = _noalloc_call(lb, plan, Qb, dt, nsteps, phys)
        assert rc == 0, lb.lib.labfm_last_error()
        torch.cuda.synchronize()
        if call > 0:  # the first call on the device may load the library's module
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        a = Qa.double().cpu().numpy()
        b = Qb.double().cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.all(_rel_l2(b, a) <= tol), (call, _rel_l2(b, a))
        assert np.all(_rel_l2(b - q_start, a - q_start) <= max(tol, 1e-10)), call
    plan.close()


def test_noalloc_rejects_plans_beyond_the_static_array(lb):
    # 3 x N x 32 bytes must fit in 16 MiB for float64: N = 180,000 does not
    ns = li.tgv_lattice(450, 400, m=2, h_over_s=1.2, jitter=0.3, seed=14)
    dev = "cuda"
    xy = torch.tensor(ns.xy, device=dev)
    h = torch.tensor(ns.h, device=dev)
    s = torch.tensor(ns.s, device=dev)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 2, residual=False)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
    Q = torch.tensor(li.tgv_fields(ns.xy, 10.0), device=dev)
    with pytest.raises(lb.LabfmError) as ei:
        lb.rk_step_noalloc(plan, Q, 1e-4, 1, lb.Phys(100.0, 0.005))
    assert ei.value.status == 4 and "static array" in str(ei.value)
    plan.close()


def test_noalloc_rejects_a_plan_of_another_device(lb):
    # a plan records the device it was built on; the static array is looked up
    # for the current device, so a mismatch is refused instead of mixing devices
    ns = li.tgv_lattice(16, 16, m=2, h_over_s=1.2, jitter=0.1, seed=15)
    dev = "cuda"
    xy = torch.tensor(ns.xy, device=dev)
    h = torch.tensor(ns.h, device=dev)
    s = torch.tensor(ns.s, device=dev)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 2, residual=False)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
    if torch.cuda.device_count() < 2:
        # one device: the check passes and the step runs
        Q = torch.tensor(li.tgv_fields(ns.xy, 10.0), device=dev)
        lb.rk_step_noalloc(plan, Q, 1e-4, 1, lb.Phys(100.0, 0.005))
        torch.cuda.synchronize()
        assert torch.isfinite(Q).all()
    else:
        with torch.cuda.device(1):
            Q = torch.tensor(li.tgv_fields(ns.xy, 10.0), device="cuda:1")
            with pytest.raises(lb.LabfmError) as ei:
                lb.rk_step_noalloc(plan, Q, 1e-4, 1, lb.Phys(100.0, 0.005))
            assert ei.value.status == 1 and "device" in str(ei.value)
    plan.close()
