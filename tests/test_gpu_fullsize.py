"""Parity at the full sizes of the variable-resolution, batched and adjoint workloads,
in the launch configurations bench.py times, on outputs the FP64 oracle can compute
row by row (sampled stencils, weights and right-hand sides), on sampled instances
of the batch, and on a directional derivative of the full-size adjoint."""
import math

import numpy as np
import pytest

import labfm_inputs as li
from oracle import core as oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, MU = 10.0, 0.005
EPS64 = np.finfo(np.float64).eps


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


def _sub_csr(rp, col, rows, N):
    """CSR over all N nodes holding only the sampled rows (others empty)."""
    cnt = np.zeros(N, dtype=np.int64)
    cnt[rows] = rp[rows + 1] - rp[rows]
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    return np.concatenate([[0], np.cumsum(cnt)]), col[idx], idx


# ---------------------------------------------------------------- variable resolution, m = 10

@pytest.fixture(scope="module")
def c3(lb):
    ns = li.varres_columns()
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 10)
    rows = np.random.default_rng(3).choice(ns.N, size=48, replace=False)
    rows = np.unique(np.concatenate([[0, ns.N - 1], rows]))
    return dict(ns=ns, s=s, rp=rp, col=col, wb=wb, rows=rows)


def test_varres_stencils_and_weights_sampled(c3):
    ns, rows = c3["ns"], c3["rows"]
    rp, col = c3["rp"].cpu().numpy(), c3["col"].cpu().numpy()
    assert ns.N > 1_000_000 - 1000 and int(c3["wb"]["status"].abs().sum().item()) == 0
    for i in rows:
        ref = oracle.neighbours_of(ns.xy, ns.h, int(i), ns.Lx, ns.Ly)
        assert np.array_equal(col[rp[i]:rp[i + 1]], ref)
    rp_r = np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])])
    col_r = np.concatenate([col[rp[i]:rp[i + 1]] for i in rows])
    ow = oracle.build_weights(ns.xy, ns.h, ns.s, rp_r, col_r, 10, ns.Lx, ns.Ly, rows=rows,
                              want_cond=True)
    wg = c3["wb"]["w"].cpu().numpy()
    n = oracle.n_unknowns(10)
    for k, i in enumerate(rows):
        wo = ow["w"][:, rp_r[k]:rp_r[k + 1]]
        err = (np.abs(wg[:, rp[i]:rp[i + 1]] - wo) / np.abs(wo).max(axis=1, keepdims=True)).max()
        assert err <= max(50 * n * EPS64 * ow["cond1"][k], 1e-13), (i, err, ow["cond1"][k])


def test_varres_rhs_sampled_fp64_and_fp32(lb, c3):
    ns, rows = c3["ns"], c3["rows"]
    rp, col = c3["rp"].cpu().numpy(), c3["col"].cpu().numpy()
    wg = c3["wb"]["w"].cpu().numpy()
    q = li.tgv_fields(ns.xy, C)
    rps, cols, idx = _sub_csr(rp, col, rows, ns.N)
    Ro = oracle.rhs(q, wg[:5, idx], rps, cols, C * C, MU)
    phys = lb.Phys(C * C, MU)
    # FP32: the elementwise rounding budget of the FP32 tests, on the sampled rows
    from test_gpu_fp32 import rhs_bound
    B = rhs_bound(q, wg[:, idx], rps, cols, C * C, MU)
    for dtype in (torch.float64, torch.float32):
        plan = lb.Plan(c3["rp"], c3["col"], c3["wb"]["w"], c3["wb"]["kappa"], c3["s"], dtype=dtype)
        # the shapes the step tuner picks for this workload: 4 lanes per node with the
        # record prefetch (the F32 plan default here), and 8 lanes
        for g in (4, 8):
            plan.set_launch(g, 128)
            R = lb.rhs(plan, _dev(q, dtype), phys).double().cpu().numpy()
            if dtype == torch.float64:
                for f in range(3):
                    err = np.abs(R[f][rows] - Ro[f][rows]).max() / np.abs(Ro[f][rows]).max()
                    assert err <= 1e-12, (f, err)
            else:
                assert plan.info()["prefetch"] == 2
                ratio = np.abs(R[:, rows] - Ro[:, rows]) / B[:, rows]
                assert ratio.max() <= 1.0, ratio.max()
        plan.close()


# ---------------------------------------------------------------- batch of 256 instances

@pytest.fixture(scope="module")
def c4(lb):
    inst = []
    for ns in li.batch_instances(256):
        d = {"ns": ns, "xy": _dev(ns.xy), "h": _dev(ns.h), "s": _dev(ns.s)}
        d["row_ptr"], d["col"] = lb.build_stencils(d["xy"], d["h"], ns.Lx, ns.Ly)
        wb = lb.build_weights(d["xy"], d["h"], d["s"], ns.Lx, ns.Ly, d["row_ptr"], d["col"], ns.m,
                              residual=False)
        d["w"], d["kappa"] = wb["w"], wb["kappa"]
        inst.append(d)
    return inst


def test_batch256_sampled_instances(lb, c4):
    inst = c4
    assert len(inst) == 256
    plan = lb.Plan.batched(inst, dtype=torch.float32)
    q0 = torch.cat([_dev(li.tgv_fields(d["ns"].xy, C), torch.float32) for d in inst], dim=1).contiguous()
    s_all = torch.cat([d["s"] for d in inst])
    dt_inst = plan.stable_dt_instances(q0, s_all, C, MU).cpu().numpy()
    plan.set_dt(dt_inst)
    plan.set_persistent(True)  # the configuration the bench's tuner picks for the batch
    phys = lb.Phys(C * C, MU)
    graph = lb.StepGraph(plan, 0.0, phys)
    Q = q0.clone()
    graph.run(Q, 2)
    graph.close()
    got = Q.double().cpu().numpy()
    off = plan.offsets
    for k in np.random.default_rng(4).choice(256, size=4, replace=False):
        d = inst[k]
        ns = d["ns"]
        q = li.tgv_fields(ns.xy, C)
        assert dt_inst[k] == pytest.approx(oracle.stable_dt(q, ns.s, C, MU), rel=1e-6)
        alone = lb.Plan(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], dtype=torch.float32)
        Qa = _dev(q, torch.float32)
        lb.rk_step(alone, Qa, float(dt_inst[k]), 2, phys)
        ref = Qa.double().cpu().numpy()
        g = got[:, off[k]:off[k + 1]]
        err = np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.all(err <= 1e-6), (k, err)
        alone.close()
    plan.close()


# ---------------------------------------------------------------- adjoint at 262,144 nodes

def test_adjoint_fullsize_directional_derivative(lb):
    # the adjoint workload's node set and initial state (512^2, m = 8, TGV + 0.05 x
    # band-limited perturbation), FP64, 40 steps with checkpoints every 10
    ns = li.tgv_lattice(512, m=8, h_over_s=2.8, jitter=0.05, seed=5)
    xy, h, s = _dev(ns.xy), _dev(ns.h), _dev(ns.s)
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 8, residual=False)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=torch.float64)
    lb.enable_adjoint(plan)
    q0 = li.perturbed_tgv_fields(ns.xy, C, amplitude=0.05, kmax=8)
    c0 = _dev(oracle.primitive_to_conserved(q0))
    dt = oracle.stable_dt(q0, ns.s, C, MU)
    phys = lb.Phys(C * C, MU)
    nsteps = 40
    c = c0.clone().requires_grad_(True)
    qf = lb.rollout(plan, lb.to_primitive(c), dt, nsteps, phys, checkpoint_every=10)
    ke = lb.domain_kinetic_energy(qf, s)
    ke.backward()
    grad = c.grad.detach()
    assert torch.isfinite(grad).all()

    def J(cc):
        q = lb.conserved_to_primitive(cc)
        lb.rk_step(plan, q, dt, nsteps, phys)
        return float(lb.kinetic_energy(q, s).item())

    v = _dev(np.random.default_rng(6).standard_normal((3, ns.N)))
    eps = 1e-6
    fd = (J(c0 + eps * v) - J(c0 - eps * v)) / (2 * eps)
    ad = float((grad * v).sum().item())
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    assert math.isfinite(float(ke.item()))
    plan.close()
