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
