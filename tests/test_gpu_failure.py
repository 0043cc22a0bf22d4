"""Failure detection on the GPU without faulting it: a bounded device-side wait
that runs out reports LABFM_ETIMEOUT through the plan's status word and leaves
the context usable; injected host-side faults (LABFM_FAULT) surface as the
status codes and node flags of the real failures."""
import numpy as np
import pytest

import labfm_inputs as li

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


def _inputs(lb, ns):
    xy = torch.tensor(ns.xy, device="cuda")
    h = torch.tensor(ns.h, device="cuda")
    s = torch.tensor(ns.s, device="cuda")
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    return xy, h, s, rp, col


def test_staged_wait_runs_out_and_reports_timeout(lb):
    ns = li.tgv_lattice(64, 48, m=8, jitter=0.05, seed=81)
    xy, h, s, rp, col = _inputs(lb, ns)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 8, residual=False)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float32)
    q0 = torch.tensor(li.tgv_fields(ns.xy, C), dtype=torch.float32, device="cuda")
    dt = float(lb.stable_dt(plan, q0, s, C, MU).item())
    phys = lb.Phys(C * C, MU)
    plan.set_launch(16, 128)
    ref = q0.clone()
    lb.rk_step(plan, ref, dt, 2, phys)  # unstaged, 16 lanes per node
    plan.set_staging(3)
    assert plan.device_status() == 0
    # a zero limit makes every wait a single non-blocking test of a copy that has
    # just been issued: the waits run out, the kernel records the timeout and returns
    plan.set_wait_limit(0)
    Q = q0.clone()
    lb.rk_step(plan, Q, dt, 1, phys)
    assert plan.device_status() == 7  # LABFM_ETIMEOUT
    assert plan.device_status() == 0  # the query clears it
    # the context is still usable: with the default limit the staged step runs and
    # equals the unstaged one bit for bit
    plan.set_wait_limit(1_000_000_000)
    Q = q0.clone()
    lb.rk_step(plan, Q, dt, 2, phys)
    assert plan.device_status() == 0
    assert torch.equal(Q, ref)
    with pytest.raises(lb.LabfmError):
        plan.set_wait_limit(-1)
    plan.close()


def test_injected_singular_node_is_flagged_and_counted(lb, monkeypatch):
    ns = li.tgv_lattice(24, 20, m=4, jitter=0.1, seed=82)
    xy, h, s, rp, col = _inputs(lb, ns)
    clean = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4, check=True)
    monkeypatch.setenv("LABFM_FAULT", "singular_node:37")
    with pytest.raises(lb.LabfmError) as ei:
        lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4, check=True)
    assert ei.value.status == 5 and "1 node(s) failed" in str(ei.value)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4)
    st = wb["status"].cpu().numpy()
    assert st[37] == 2 and np.count_nonzero(st) == 1  # LABFM_NODE_SINGULAR on node 37 only
    # nothing else changes
    assert torch.equal(wb["w"], clean["w"]) and torch.equal(wb["kappa"], clean["kappa"])
    # a node beyond N is not flagged
    monkeypatch.setenv("LABFM_FAULT", f"singular_node:{ns.N}")
    assert lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4, check=True)["n_failed"] == 0


def test_injected_allocation_failure_leaves_device_memory_alone(lb, monkeypatch):
    ns = li.tgv_lattice(24, 20, m=4, jitter=0.1, seed=83)
    xy, h, s, rp, col = _inputs(lb, ns)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("LABFM_FAULT", "alloc")
    with pytest.raises(lb.LabfmError) as ei:
        lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
    assert ei.value.status == 3 and "injected" in str(ei.value)
    with pytest.raises(lb.LabfmError) as ei:
        lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    assert ei.value.status == 3
    assert torch.cuda.mem_get_info()[0] == free0
    monkeypatch.delenv("LABFM_FAULT")
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
    Q = torch.tensor(li.tgv_fields(ns.xy, C), device="cuda")
    lb.rk_step(plan, Q, 1e-4, 1, lb.Phys(C * C, MU))
    assert torch.isfinite(Q).all()
    plan.close()


def test_state_check_reports_a_diverging_run(lb):
    # the +-0.3 s lattice without node shifting goes non-finite within tens of steps
    # (the filter amplifies a few modes); with the state check on, the run reports
    # LABFM_ENONFINITE, and a finite run on the +-0.05 s lattice reports nothing
    phys = lb.Phys(C * C, MU)
    for jitter, diverges in ((0.3, True), (0.05, False)):
        ns = li.tgv_lattice(64, m=4, h_over_s=1.7, jitter=jitter, seed=0)
        xy, h, s, rp, col = _inputs(lb, ns)
        wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4, residual=False)
        for dtype in (torch.float64, torch.float32):
            plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
            Q = torch.tensor(li.tgv_fields(ns.xy, C), dtype=dtype, device="cuda")
            dt = float(lb.stable_dt(plan, Q, s, C, MU).item())
            plan.set_check_finite(25)
            lb.rk_step(plan, Q, dt, 300, phys)
            finite = bool(torch.isfinite(Q).all().item())
            status = plan.device_status()
            assert finite != diverges, (jitter, dtype)
            assert status == (6 if diverges else 0), (jitter, dtype, status)  # LABFM_ENONFINITE
            assert plan.device_status() == 0  # the query clears it
            # turned off, the same run reports nothing
            plan.set_check_finite(0)
            Q = torch.tensor(li.tgv_fields(ns.xy, C), dtype=dtype, device="cuda")
            lb.rk_step(plan, Q, dt, 300, phys)
            assert plan.device_status() == 0
            with pytest.raises(lb.LabfmError):
                plan.set_check_finite(-1)
            plan.close()


def test_injected_timeout_is_reported(lb, monkeypatch):
    ns = li.tgv_lattice(24, 20, m=4, jitter=0.1, seed=84)
    xy, h, s, rp, col = _inputs(lb, ns)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 4)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float32)
    assert plan.device_status() == 0
    monkeypatch.setenv("LABFM_FAULT", "timeout")
    assert plan.device_status() == 7  # LABFM_ETIMEOUT, as a bounded wait that ran out
    monkeypatch.delenv("LABFM_FAULT")
    assert plan.device_status() == 0
    # an injected allocation failure of the status word
    monkeypatch.setenv("LABFM_FAULT", "alloc")
    with pytest.raises(lb.LabfmError) as ei:
        plan.set_check_finite(5)
    assert ei.value.status == 3
    monkeypatch.delenv("LABFM_FAULT")
    plan.set_check_finite(5)
    plan.close()
