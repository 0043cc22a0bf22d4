"""Boundaries on batched plans (Section 7.1): channels between no-slip walls and open
boxes with an inflow and an outflow, batched with their boundary nodes given in the
plan's numbering, evolve bit for bit as each instance does alone, with plain launches
and inside a captured step graph, also with a launch range per interior order."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import boundary_oracle as bo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, MU = 10.0, 0.01


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


def _instance(lb, ns, periodic, seed):
    cols, normals = li.channel_walls(ns)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    op = lb.build_wall_operator(xy, h, s, ns.Lx, ns.Ly, ns.m, 4, _dev(cols, torch.int32), _dev(normals),
                                periodic=periodic, check=True)
    q0 = np.zeros((3, ns.N))
    q0[0] = 0.01 * li.smooth_perturbation(ns.xy, kmax=3, seed=seed, Lx=ns.Lx, Ly=ns.Ly)
    q0[1] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=seed + 1, Lx=ns.Lx, Ly=ns.Ly)
    q0[2] = 0.1 * li.smooth_perturbation(ns.xy, kmax=3, seed=seed + 2, Lx=ns.Lx, Ly=ns.Ly)
    return dict(ns=ns, row_ptr=op["row_ptr"], col=op["col"], w=op["w"], kappa=op["kappa"], s=s,
                nodes=cols[:, 0].astype(np.int32), normal=normals, q0=q0)


def _run(lb, plan, q0, dt, nsteps, phys, graph, dtype):
    Q = _dev(q0, dtype)
    if graph:
        gr = lb.StepGraph(plan, dt, phys)
        gr.run(Q, nsteps)
        gr.close()
    else:
        lb.rk_step(plan, Q, dt, nsteps, phys)
    return Q.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("graph", [False, True])
def test_batched_channels_match_channels_alone(lb, dtype, graph):
    inst = [_instance(lb, li.channel(24, 20, m=6, jitter=0.1, seed=91), (True, False), 5),
            _instance(lb, li.channel(30, 16, m=6, jitter=0.1, seed=92), (True, False), 9)]
    for d in inst:
        d["q0"][1:, d["nodes"]] = 0.0
    phys = lb.Phys(C * C, MU, 0.5, 0.0)
    nsteps = 4
    alone, dts = [], []
    for d in inst:
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        plan.set_walls(_dev(d["nodes"], torch.int32), _dev(d["normal"]))
        dt = 0.25 * float(lb.stable_dt(plan, _dev(np.stack([d["q0"][0], d["q0"][1] + 1.0, d["q0"][2]]), dtype),
                                       d["s"], C, MU).item())
        dts.append(dt)
        alone.append(_run(lb, plan, d["q0"], dt, nsteps, phys, graph, dtype))
        plan.close()
    bp = lb.Plan.batched(inst, dtype=dtype)
    off = bp.offsets
    bp.set_walls(_dev(np.concatenate([d["nodes"] + off[k] for k, d in enumerate(inst)]), torch.int32),
                 _dev(np.concatenate([d["normal"] for d in inst])))
    bp.set_dt(dts)
    got = _run(lb, bp, np.concatenate([d["q0"] for d in inst], axis=1), 0.0, nsteps, phys, graph, dtype)
    for k, d in enumerate(inst):
        part = got[:, off[k]:off[k + 1]]
        assert np.all(np.isfinite(part))
        assert np.all(part[1:, d["nodes"]] == 0.0)
        assert np.array_equal(part, alone[k]), k
    bp.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_channels_of_two_orders_with_launch_ranges(lb, dtype):
    # interior orders m = 6 and 4, each class its own launch range and shape: every
    # instance evolves as it does alone in that shape
    inst = [_instance(lb, li.channel(26, 18, m=4, jitter=0.1, seed=95), (True, False), 21),
            _instance(lb, li.channel(24, 20, m=6, jitter=0.1, seed=96), (True, False), 25)]
    shapes = [(2, 0), (4, 2)]
    for d in inst:
        d["q0"][1:, d["nodes"]] = 0.0
    phys = lb.Phys(C * C, MU, 0.5, 0.0)
    alone, dts = [], []
    for d, (g, pf) in zip(inst, shapes):
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        plan.set_walls(_dev(d["nodes"], torch.int32), _dev(d["normal"]))
        plan.set_launch(g, 128)
        plan.set_prefetch(pf if dtype == torch.float32 else 0)
        dt = 0.25 * float(lb.stable_dt(plan, _dev(np.stack([d["q0"][0], d["q0"][1] + 1.0, d["q0"][2]]), dtype),
                                       d["s"], C, MU).item())
        dts.append(dt)
        alone.append(_run(lb, plan, d["q0"], dt, 3, phys, False, dtype))
        plan.close()
    bp = lb.Plan.batched(inst, dtype=dtype)
    off = bp.offsets
    bp.set_walls(_dev(np.concatenate([d["nodes"] + off[k] for k, d in enumerate(inst)]), torch.int32),
                 _dev(np.concatenate([d["normal"] for d in inst])))
    bp.set_dt(dts)
    bp.set_launch_ranges(off, [g for g, _ in shapes], [pf for _, pf in shapes])
    for graph in (False, True):
        got = _run(lb, bp, np.concatenate([d["q0"] for d in inst], axis=1), 0.0, 3, phys, graph, dtype)
        for k in range(len(inst)):
            assert np.array_equal(got[:, off[k]:off[k + 1]], alone[k]), (k, graph)
    bp.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_open_boxes_match_boxes_alone(lb, dtype):
    inst = [_instance(lb, li.open_box(28, 12, m=6, jitter=0.05, seed=93), (False, True), 13),
            _instance(lb, li.open_box(28, 12, m=6, jitter=0.05, seed=94), (False, True), 17)]
    U0 = 1.0
    for d in inst:
        nb = len(d["nodes"]) // 2
        d["kind"] = np.array([bo.INFLOW] * nb + [bo.OUTFLOW] * nb, dtype=np.int32)
        d["target"] = np.zeros((2 * nb, 2))
        d["target"][:nb, 0] = U0
        d["target"][nb:, 0] = C * C
        d["q0"][1] += U0
    params = dict(sigma=0.278, L=inst[0]["ns"].Lx, mach=U0 / C, rho0=1.0)
    phys = lb.Phys(C * C, MU)
    nsteps = 4
    alone, dts = [], []
    for d in inst:
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        plan.set_boundaries(_dev(d["nodes"], torch.int32), _dev(d["normal"]), _dev(d["kind"], torch.int32),
                            _dev(d["target"]), **params)
        dt = 0.25 * float(lb.stable_dt(plan, _dev(d["q0"], dtype), d["s"], C, MU).item())
        dts.append(dt)
        alone.append(_run(lb, plan, d["q0"], dt, nsteps, phys, False, dtype))
        plan.close()
    bp = lb.Plan.batched(inst, dtype=dtype)
    off = bp.offsets
    cat = lambda key, f=lambda k, a: a: np.concatenate([f(k, d[key]) for k, d in enumerate(inst)])
    bp.set_boundaries(_dev(cat("nodes", lambda k, a: a + off[k]), torch.int32), _dev(cat("normal")),
                      _dev(cat("kind"), torch.int32), _dev(cat("target")), **params)
    bp.set_dt(dts)
    got = _run(lb, bp, np.concatenate([d["q0"] for d in inst], axis=1), 0.0, nsteps, phys, False, dtype)
    for k in range(len(inst)):
        part = got[:, off[k]:off[k + 1]]
        assert np.all(np.isfinite(part))
        assert np.array_equal(part, alone[k]), k
    bp.close()
