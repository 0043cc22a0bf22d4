"""The F32 stage kernel with the operator stream staged through shared memory by
bulk copies: bit-identical to the unstaged kernel with the same lanes per node
(same chunk-to-lane assignment and summation order), for uniform, uneven and
batched plans, ragged node counts, every ring depth, and inside the step graph;
and one case against the FP64 oracle."""
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


def _operator(lb, ns, m):
    xy = torch.tensor(ns.xy, device="cuda")
    h = torch.tensor(ns.h, device="cuda")
    s = torch.tensor(ns.s, device="cuda")
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, m, residual=False)
    return {"row_ptr": rp, "col": col, "w": wb["w"], "kappa": wb["kappa"], "s": s, "ns": ns}


def _run(lb, plan, q0, dt, steps, group, stages, graph=False):
    plan.set_launch(group, 128)
    plan.set_staging(stages)
    Q = q0.clone()
    phys = lb.Phys(C * C, MU)
    if graph:
        g = lb.StepGraph(plan, dt, phys)
        g.run(Q, steps)
        g.close()
    else:
        lb.rk_step(plan, Q, dt, steps, phys)
    assert plan.device_status() == 0
    return Q


@pytest.fixture(scope="module")
def uniform(lb):
    # ragged node count (97 x 89) so that the last round is partly idle
    return _operator(lb, li.tgv_lattice(97, 89, m=8, jitter=0.05, seed=71), 8)


@pytest.mark.parametrize("group", [16, 32])
@pytest.mark.parametrize("stages", [2, 3, 4])
def test_staged_equals_unstaged(lb, uniform, group, stages):
    d = uniform
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    q0 = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=torch.float32, device="cuda")
    dt = float(lb.stable_dt(plan, q0, d["s"], C, MU).item())
    ref = _run(lb, plan, q0, dt, 3, group, 0)
    got = _run(lb, plan, q0, dt, 3, group, stages)
    assert torch.equal(got, ref)
    plan.close()


def test_staged_in_step_graph(lb, uniform):
    d = uniform
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    q0 = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=torch.float32, device="cuda")
    dt = float(lb.stable_dt(plan, q0, d["s"], C, MU).item())
    ref = _run(lb, plan, q0, dt, 4, 32, 0)
    got = _run(lb, plan, q0, dt, 4, 32, 3, graph=True)
    assert torch.equal(got, ref)
    plan.close()


def test_staged_uneven_stencils_and_batches(lb):
    # variable resolution m = 10 (92-221 neighbours, rounds of very different sizes)
    # batched with two small lattices of other orders
    parts = [_operator(lb, li.varres_columns(s0=0.012, m=10, seed=2), 10),
             _operator(lb, li.tgv_lattice(13, 11, m=4, jitter=0.1, seed=72), 4),
             _operator(lb, li.tgv_lattice(23, 29, m=6, jitter=0.1, seed=73), 6)]
    plan = lb.Plan.batched(parts, dtype=torch.float32)
    q0 = torch.cat([torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=torch.float32, device="cuda")
                    for d in parts], dim=1).contiguous()
    s_all = torch.cat([d["s"] for d in parts])
    plan.set_dt(plan.stable_dt_instances(q0, s_all, C, MU).cpu().tolist())
    for group in (16, 32):
        ref = _run(lb, plan, q0, 0.0, 2, group, 0)
        got = _run(lb, plan, q0, 0.0, 2, group, 4)
        assert torch.equal(got, ref)
    plan.close()


def test_staged_matches_oracle(lb):
    # one staged FP32 step against the FP64 oracle within the per-node budget of
    # one FP32 step derived in tests/fp32_budget.py (the staged kernel does the
    # unstaged kernel's arithmetic; several steps are covered by the bit-identity
    # tests above)
    from tests.fp32_budget import step_bound
    ns = li.tgv_lattice(30, 26, m=6, h_over_s=2.2, jitter=0.1, seed=74)
    d = _operator(lb, ns, 6)
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    q = li.tgv_fields(ns.xy, C)
    q0 = torch.tensor(q, dtype=torch.float32, device="cuda")
    dt = oracle.stable_dt(q, ns.s, C, MU)
    got = _run(lb, plan, q0, dt, 1, 32, 3).double().cpu().numpy()
    w, kap = d["w"].cpu().numpy(), d["kappa"].cpu().numpy()
    rp, col = d["row_ptr"].cpu().numpy(), d["col"].cpu().numpy()
    q1 = oracle.time_step(q, dt, w, kap, rp, col, C * C, MU)
    bound = step_bound(q, q1, dt, w, kap, rp, col, C * C, MU)
    ratio = np.abs(got - q1) / bound
    assert ratio.max() <= 1.0, ratio.max()
    plan.close()


def test_staging_argument_checks(lb, uniform):
    d = uniform
    p64 = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float64)
    with pytest.raises(lb.LabfmError):
        p64.set_staging(3)
    p64.set_staging(0)
    p64.close()
    p32 = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    for bad in (1, 5, -1):
        with pytest.raises(lb.LabfmError):
            p32.set_staging(bad)
    assert p32.device_status() == 0
    p32.close()


def test_prefetch_distance_changes_nothing_but_time(lb, uniform):
    # the L2 prefetch of the record stream only moves data earlier: every distance
    # gives the same bits, with the plain and the persistent kernel
    d = uniform
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    assert plan.info()["prefetch"] == 2  # the F32 default
    q0 = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=torch.float32, device="cuda")
    dt = float(lb.stable_dt(plan, q0, d["s"], C, MU).item())
    plan.set_prefetch(0)
    ref = _run(lb, plan, q0, dt, 3, 4, 0)
    for persistent in (False, True):
        plan.set_persistent(persistent)
        for pf in (1, 2, 5, 8):
            plan.set_prefetch(pf)
            assert torch.equal(_run(lb, plan, q0, dt, 3, 4, 0), ref), (persistent, pf)
    for bad in (-1, 9):
        with pytest.raises(lb.LabfmError):
            plan.set_prefetch(bad)
    plan.close()
