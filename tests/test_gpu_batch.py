"""Batched plans: many independent instances of different sizes and orders in one
plan, per-instance time steps, the persistent work-queue stage kernel, and the
per-step CUDA graph.  Each instance of a batch must evolve exactly as it does
alone, and one instance is checked against the FP64 oracle."""
import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [(20, 20, 4), (17, 23, 6), (24, 24, 8), (9, 9, 4), (31, 16, 6)]
C, MU = 10.0, 0.005


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2102_02019_gb300 as lb
    return lb


def _build_instances(lb):
    out = []
    for k, (nx, ny, m) in enumerate(SPECS):
        ns = li.tgv_lattice(nx, ny, m=m, jitter=0.1, seed=40 + k, s=1.0 / max(nx, ny))
        d = {"ns": ns}
        d["xy"] = torch.tensor(ns.xy, device="cuda")
        d["h"] = torch.tensor(ns.h, device="cuda")
        d["s"] = torch.tensor(ns.s, device="cuda")
        d["row_ptr"], d["col"] = lb.build_stencils(d["xy"], d["h"], ns.Lx, ns.Ly)
        wb = lb.build_weights(d["xy"], d["h"], d["s"], ns.Lx, ns.Ly, d["row_ptr"], d["col"], m,
                              check=True)
        d["w"], d["kappa"] = wb["w"], wb["kappa"]
        d["q0"] = li.tgv_fields(ns.xy, C)
        out.append(d)
    return out


@pytest.fixture(scope="module")
def inst(lb):
    return _build_instances(lb)


def _stack(fields):
    """3 x N_total state of a batch: instance after instance within each field."""
    return np.concatenate(fields, axis=1)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", ["plain", "persistent", "graph"])
def test_batch_matches_instances_alone(lb, inst, dtype, mode):
    phys = lb.Phys(C * C, MU)
    nsteps = 3
    alone = []
    dts = []
    for d in inst:
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        Q = torch.tensor(d["q0"], dtype=dtype, device="cuda")
        dt = float(lb.stable_dt(plan, Q, d["s"], C, MU).item())
        dts.append(dt)
        lb.rk_step(plan, Q, dt, nsteps, phys)
        alone.append(Q.double().cpu().numpy())
        plan.close()
    bplan = lb.Plan.batched(inst, dtype=dtype)
    assert bplan.info()["n_instances"] == len(inst)
    Qb = torch.tensor(_stack([d["q0"] for d in inst]), dtype=dtype, device="cuda")
    s_all = torch.cat([d["s"] for d in inst])
    dt_inst = bplan.stable_dt_instances(Qb, s_all, C, MU).cpu().numpy()
    assert np.array_equal(dt_inst, np.array(dts))  # exact minimum per instance
    bplan.set_dt(dt_inst)
    if mode == "persistent":
        bplan.set_persistent(True)
    if mode == "graph":
        bplan.set_persistent(True)
        graph = lb.StepGraph(bplan, 0.0, phys)
        graph.run(Qb, nsteps)
        graph.close()
    else:
        lb.rk_step(bplan, Qb, 0.0, nsteps, phys)
    got = Qb.double().cpu().numpy()
    off = bplan.offsets
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    for k, a in enumerate(alone):
        g = got[:, off[k]:off[k + 1]]
        err = np.linalg.norm(g - a, axis=1) / np.linalg.norm(a, axis=1)
        assert np.all(err <= tol), (k, err)
    bplan.close()


def test_batch_instance_matches_oracle(lb, inst):
    # the m = 8 instance of the batch, FP64, against the oracle with GPU-built weights
    k = 2
    d = inst[k]
    phys = lb.Phys(C * C, MU)
    bplan = lb.Plan.batched(inst, dtype=torch.float64)
    Qb = torch.tensor(_stack([e["q0"] for e in inst]), device="cuda")
    s_all = torch.cat([e["s"] for e in inst])
    dt_inst = bplan.stable_dt_instances(Qb, s_all, C, MU).cpu().numpy()
    bplan.set_dt(dt_inst)
    bplan.set_persistent(True)
    lb.rk_step(bplan, Qb, 0.0, 2, phys)
    got = Qb.cpu().numpy()[:, bplan.offsets[k]:bplan.offsets[k + 1]]
    ns = d["ns"]
    rp = d["row_ptr"].cpu().numpy()
    col = d["col"].cpu().numpy()
    w = d["w"].cpu().numpy()
    kap = d["kappa"].cpu().numpy()
    q = d["q0"]
    assert dt_inst[k] == oracle.stable_dt(q, ns.s, C, MU)
    for _ in range(2):
        q = oracle.time_step(q, dt_inst[k], w, kap, rp, col, C * C, MU)
    err = np.linalg.norm(got - q, axis=1) / np.linalg.norm(q, axis=1)
    assert np.all(err <= 1e-12), err
    bplan.close()


def test_persistent_handles_uneven_stencils(lb):
    # variable stencil sizes (h varies 0.85..1.25 around 3.3 s, m = 10) in one plan
    ns = li.varres_columns(s0=0.012, m=10, seed=2)
    xy = torch.tensor(ns.xy, device="cuda")
    h = torch.tensor(ns.h, device="cuda")
    s = torch.tensor(ns.s, device="cuda")
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    counts = np.diff(rp.cpu().numpy())
    assert counts.min() > 65 and counts.max() > 1.8 * counts.min()
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 10, check=True)
    phys = lb.Phys(C * C, MU)
    q0 = torch.tensor(li.tgv_fields(ns.xy, C), device="cuda")
    out = []
    for persistent in (False, True):
        plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
        plan.set_persistent(persistent)
        Q = q0.clone()
        lb.rk_step(plan, Q, 1e-4, 2, phys)
        out.append(Q.cpu().numpy())
        plan.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("graph", [False, True])
def test_launch_ranges_match_instances_alone_with_their_shapes(lb, inst, dtype, graph):
    # instances grouped by order, one launch range per order class with its own
    # lanes per node and prefetch: every instance evolves bit for bit as it does
    # alone with that range's shape
    order = sorted(range(len(inst)), key=lambda k: inst[k]["ns"].m)
    grouped = [inst[k] for k in order]
    shapes = {4: (2, 0), 6: (8, 2), 8: (4, 2)}
    phys = lb.Phys(C * C, MU)
    nsteps = 3
    alone, dts = [], []
    for d in grouped:
        plan = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=dtype)
        g, pf = shapes[d["ns"].m]
        plan.set_launch(g, 128)
        plan.set_prefetch(pf if dtype == torch.float32 else 0)
        Q = torch.tensor(d["q0"], dtype=dtype, device="cuda")
        dt = float(lb.stable_dt(plan, Q, d["s"], C, MU).item())
        dts.append(dt)
        lb.rk_step(plan, Q, dt, nsteps, phys)
        alone.append(Q.double().cpu().numpy())
        plan.close()
    bplan = lb.Plan.batched(grouped, dtype=dtype)
    bplan.set_dt(dts)
    off = bplan.offsets
    classes = []
    for m in (4, 6, 8):
        ks = [k for k, d in enumerate(grouped) if d["ns"].m == m]
        classes.append((off[ks[0]], off[ks[-1] + 1], m))
    bplan.set_launch_ranges([c[0] for c in classes] + [classes[-1][1]],
                            [shapes[c[2]][0] for c in classes], [shapes[c[2]][1] for c in classes])
    Qb = torch.tensor(_stack([d["q0"] for d in grouped]), dtype=dtype, device="cuda")
    if graph:
        gr = lb.StepGraph(bplan, 0.0, phys)
        gr.run(Qb, nsteps)
        gr.close()
    else:
        lb.rk_step(bplan, Qb, 0.0, nsteps, phys)
    got = Qb.double().cpu().numpy()
    for k, d in enumerate(grouped):
        assert np.array_equal(got[:, off[k]:off[k + 1]], alone[k]), k
    # argument checks, and removing the ranges
    with pytest.raises(lb.LabfmError):
        bplan.set_launch_ranges([0, 5], [4], [2])  # does not cover [0, N)
    with pytest.raises(lb.LabfmError):
        bplan.set_launch_ranges([0, bplan.N], [3], [2])  # unsupported lanes per node
    bplan.set_launch_ranges([], [], [])
    assert bplan.info()["n_instances"] == len(grouped)
    bplan.close()


def test_range_tuner_and_cache(lb, inst, tmp_path, monkeypatch):
    # the per-class tuner picks a supported shape for every class, writes its cache,
    # and a second plan reads the shapes from it without timing
    monkeypatch.setenv("LABFM_TUNE_CACHE", str(tmp_path / "tune.json"))
    order = sorted(range(len(inst)), key=lambda k: inst[k]["ns"].m)
    grouped = [inst[k] for k in order]
    bplan = lb.Plan.batched(grouped, dtype=torch.float32)
    Q = torch.tensor(_stack([d["q0"] for d in grouped]), dtype=torch.float32, device="cuda")
    s_all = torch.cat([d["s"] for d in grouped])
    bplan.set_dt(bplan.stable_dt_instances(Q, s_all, C, MU).cpu().numpy())
    off = bplan.offsets
    classes = []
    for m in (4, 6, 8):
        ks = [k for k, d in enumerate(grouped) if d["ns"].m == m]
        nnz = sum(grouped[k]["col"].numel() for k in ks)
        classes.append((off[ks[0]], off[ks[-1] + 1], m, nnz / (off[ks[-1] + 1] - off[ks[0]])))
    first = bplan.tune_ranges(Q, lb.Phys(C * C, MU), 0.0, classes, steps=1)
    assert all(c["group"] in (2, 4, 8, 16) and not c["from_cache"] for c in first)
    assert (tmp_path / "tune.json").exists()
    second = bplan.tune_ranges(Q, lb.Phys(C * C, MU), 0.0, classes, steps=1)
    assert all(c["from_cache"] for c in second)
    assert [(c["group"], c["prefetch"]) for c in first] == [(c["group"], c["prefetch"]) for c in second]
    bplan.close()
