"""Programmatic dependent launches change the schedule, not the arithmetic: with
them on (the default) and off, time steps, batched steps with per-order launch
ranges in a captured step graph, walls, and the recorded adjoint step give the
same state bit for bit."""
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


def _operator(lb, nx, ny, m, seed):
    # a ragged node count (not a multiple of the 32-node blocks) with jitter
    ns = li.tgv_lattice(nx, ny, m=m, jitter=0.1, seed=seed, s=1.0 / max(nx, ny))
    xy, h, s = (torch.tensor(a, device="cuda") for a in (ns.xy, ns.h, ns.s))
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, m, check=True)
    return dict(ns=ns, row_ptr=rp, col=col, w=wb["w"], kappa=wb["kappa"], s=s)


@pytest.fixture(scope="module")
def ops(lb):
    return [_operator(lb, 45, 38, 8, 71), _operator(lb, 33, 29, 4, 72), _operator(lb, 40, 41, 6, 73)]


def _step(lb, d, dtype, programmatic, nsteps=4, group=4):
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
    plan.set_programmatic_launch(programmatic)
    assert plan.info()["programmatic"] == int(programmatic)
    plan.set_launch(group, 128)
    Q = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=dtype, device="cuda")
    dt = float(lb.stable_dt(plan, Q, d["s"], C, MU).item())
    lb.rk_step(plan, Q, dt, nsteps, lb.Phys(C * C, MU))
    plan.close()
    return Q


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("group", [2, 4, 16])
def test_time_steps_equal_with_and_without(lb, ops, dtype, group):
    for d in ops:
        a = _step(lb, d, dtype, True, group=group)
        b = _step(lb, d, dtype, False, group=group)
        assert torch.isfinite(a).all()
        assert torch.equal(a, b), (d["ns"].N, dtype, group)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_ranges_in_a_step_graph_equal_with_and_without(lb, ops, dtype):
    order = sorted(range(len(ops)), key=lambda k: ops[k]["ns"].m)
    grouped = [ops[k] for k in order]
    phys = lb.Phys(C * C, MU)
    dts = []
    for d in grouped:
        p = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        q = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=dtype, device="cuda")
        dts.append(float(lb.stable_dt(p, q, d["s"], C, MU).item()))
        p.close()
    q0 = np.concatenate([li.tgv_fields(d["ns"].xy, C) for d in grouped], axis=1)
    out = []
    for programmatic in (True, False):
        bp = lb.Plan.batched(grouped, dtype=dtype)
        bp.set_programmatic_launch(programmatic)
        bp.set_dt(dts)
        off = bp.offsets
        bp.set_launch_ranges(off, [2, 8, 4], [0, 2, 2])
        Q = torch.tensor(q0, dtype=dtype, device="cuda")
        gr = lb.StepGraph(bp, 0.0, phys)
        gr.run(Q, 3)
        gr.close()
        lb.rk_step(bp, Q, 0.0, 2, phys)
        out.append(Q)
        bp.close()
    assert torch.isfinite(out[0]).all()
    assert torch.equal(out[0], out[1])


def test_walls_equal_with_and_without(lb):
    ns = li.channel(24, 20, m=6, jitter=0.1, seed=74)
    cols, normals = li.channel_walls(ns)
    xy, h, s = (torch.tensor(a, device="cuda") for a in (ns.xy, ns.h, ns.s))
    op = lb.build_wall_operator(xy, h, s, ns.Lx, ns.Ly, 6, 4, torch.tensor(cols, device="cuda"),
                                torch.tensor(normals, device="cuda"), periodic=(True, False), check=True)
    q0 = np.zeros((3, ns.N))
    q0[1] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=11, Ly=ns.Ly)
    q0[1:, cols[:, 0]] = 0.0
    out = []
    for programmatic in (True, False):
        plan = lb.Plan(op["row_ptr"], op["col"], op["w"], op["kappa"], s, dtype=torch.float32)
        plan.set_programmatic_launch(programmatic)
        plan.set_walls(torch.tensor(cols[:, 0], device="cuda"), torch.tensor(normals, device="cuda"))
        Q = torch.tensor(q0, dtype=torch.float32, device="cuda")
        lb.rk_step(plan, Q, 1e-4, 4, lb.Phys(C * C, 0.01, 0.5, 0.0))
        out.append(Q)
        plan.close()
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_recorded_adjoint_step_equal_with_and_without(lb, ops, dtype):
    d = ops[0]
    phys = lb.Phys(C * C, MU)
    res = []
    for programmatic in (True, False):
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        plan.set_programmatic_launch(programmatic)
        lb.enable_adjoint(plan)
        Q = torch.tensor(li.tgv_fields(d["ns"].xy, C), dtype=dtype, device="cuda")
        dt = float(lb.stable_dt(plan, Q, d["s"], C, MU).item())
        states = lb.stage_states(plan)
        lb.rk_step_record(plan, Q, states, dt, phys)
        lam = torch.tensor(np.cos(3.0 * d["ns"].xy[:, 0])[None, :] * np.ones((3, 1)), dtype=dtype, device="cuda")
        lb.rk_step_adjoint_recorded(plan, states, lam, dt, phys)
        g = lb.rhs_adjoint(plan, Q, lam.clone(), phys)
        res.append((Q, lam, g))
        plan.close()
    for a, b in zip(res[0], res[1]):
        assert torch.isfinite(a).all()
        assert torch.equal(a, b)


def test_setting_is_checked(lb, ops):
    d = ops[1]
    plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
    assert plan.info()["programmatic"] == 1
    assert lb.lib.labfm_plan_set_programmatic_launch(plan.handle, 2) == 1
    assert lb.lib.labfm_plan_set_programmatic_launch(None, 1) != 0
    plan.close()
