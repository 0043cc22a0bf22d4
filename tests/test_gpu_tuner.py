"""The step tuner (Plan.tune_step): it leaves the state alone, leaves the plan in the
shape it reports, and a plan set to that shape by hand steps to the same state bit
for bit."""
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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_tuned_shape_is_applied_and_reproducible(lb, dtype):
    ns = li.tgv_lattice(40, 36, m=6, jitter=0.1, seed=81, s=1.0 / 40)
    xy, h, s = (torch.tensor(a, device="cuda") for a in (ns.xy, ns.h, ns.s))
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, ns.m, check=True)
    phys = lb.Phys(C * C, MU)
    plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
    Q = torch.tensor(li.tgv_fields(ns.xy, C), dtype=dtype, device="cuda")
    Q0 = Q.clone()
    dt = float(lb.stable_dt(plan, Q, s, C, MU).item())
    cfg = plan.tune_step(Q, phys, dt, steps=1, groups=(2, 4, 8), staged=(), prefetch=(0, 2),
                         filter_groups=(2, 4), filter_blocks=(64, 128))
    assert torch.equal(Q, Q0)
    info = plan.info()
    assert (info["group"], info["block"], info["filter_group"], info["filter_persistent"]) == \
        (cfg["group"], cfg["block"], cfg["filter_group"], int(cfg["filter_persistent"]))
    # the filter keeps the plan's own lanes per node when no filter shape was faster
    assert cfg["block"] in (64, 128) and cfg["group"] in (2, 4, 8) and cfg["filter_group"] in (2, 4, cfg["group"])
    if dtype == torch.float32:
        assert info["prefetch"] == cfg["prefetch"]
    lb.rk_step(plan, Q, dt, 3, phys)
    # the same shape set by hand on a fresh plan
    ref = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
    ref.set_persistent(cfg["persistent"])
    ref.set_staging(0)
    if dtype == torch.float32:
        ref.set_prefetch(cfg["prefetch"])
    ref.set_launch(cfg["group"], cfg["block"])
    ref.set_filter_launch(cfg["filter_group"], cfg["filter_persistent"])
    Qr = Q0.clone()
    lb.rk_step(ref, Qr, dt, 3, phys)
    assert torch.isfinite(Q).all()
    assert torch.equal(Q, Qr)
    plan.close()
    ref.close()
