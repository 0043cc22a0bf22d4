"""Checkpoint and resume on the host: a built operator and an evolved state written
to .npz and read back unchanged (bit for bit, dtypes kept), with their metadata."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2102_02019_gb300 as lb
    return lb


def test_operator_round_trip(lb, tmp_path):
    rng = np.random.default_rng(0)
    N, nnz = 37, 211
    row_ptr = torch.tensor(np.sort(np.concatenate([[0, nnz], rng.integers(0, nnz, N - 1)])), dtype=torch.int32)
    col = torch.tensor(rng.integers(0, N, nnz), dtype=torch.int32)
    w = torch.tensor(rng.standard_normal((6, nnz)))
    kappa = torch.tensor(rng.standard_normal(N))
    s = torch.tensor(rng.uniform(0.01, 0.02, N))
    p = tmp_path / "op.npz"
    lb.save_operator(str(p), row_ptr, col, w, kappa, s, m=8, h_over_s=2.8, workload="test")
    got = lb.load_operator(str(p), device="cpu")
    for k, t in (("row_ptr", row_ptr), ("col", col), ("w", w), ("kappa", kappa), ("s", s)):
        assert got[k].dtype == t.dtype and torch.equal(got[k], t), k
    assert got["meta"] == {"m": 8, "h_over_s": 2.8, "workload": "test"}


def test_state_round_trip(lb, tmp_path):
    Q = torch.tensor(np.random.default_rng(1).standard_normal((3, 101)), dtype=torch.float32)
    p = tmp_path / "state.npz"
    lb.save_state(str(p), Q, step=250, t=0.125, dt=5e-4, seed=7)
    got = lb.load_state(str(p), device="cpu")
    assert got["Q"].dtype == torch.float32 and torch.equal(got["Q"], Q)
    assert (got["step"], got["t"], got["dt"], got["meta"]) == (250, 0.125, 5e-4, {"seed": 7})


@pytest.mark.gpu
def test_resume_from_checkpoint_is_bit_identical(lb, tmp_path):
    # 20 steps in one go equal 10 steps, a checkpoint of the operator and the state,
    # a fresh plan from the reloaded operator, and 10 more steps
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import labfm_inputs as li
    ns = li.tgv_lattice(48, m=6, h_over_s=2.2, jitter=0.05, seed=3)
    xy, h, s = (torch.tensor(a, device="cuda") for a in (ns.xy, ns.h, ns.s))
    rp, col = lb.build_stencils(xy, h, ns.Lx, ns.Ly)
    wb = lb.build_weights(xy, h, s, ns.Lx, ns.Ly, rp, col, 6)
    phys = lb.Phys(100.0, 0.005)
    for dtype in (torch.float64, torch.float32):
        plan = lb.Plan(rp, col, wb["w"], wb["kappa"], s, dtype=dtype)
        Q0 = torch.tensor(li.tgv_fields(ns.xy, 10.0), dtype=dtype, device="cuda")
        dt = float(lb.stable_dt(plan, Q0, s, 10.0, 0.005).item())
        ref = Q0.clone()
        lb.rk_step(plan, ref, dt, 20, phys)
        Q = Q0.clone()
        lb.rk_step(plan, Q, dt, 10, phys)
        lb.save_operator(str(tmp_path / "op.npz"), rp, col, wb["w"], wb["kappa"], s, m=6)
        lb.save_state(str(tmp_path / "q.npz"), Q, step=10, t=10 * dt, dt=dt)
        plan.close()
        op = lb.load_operator(str(tmp_path / "op.npz"))
        st = lb.load_state(str(tmp_path / "q.npz"))
        plan2 = lb.Plan(op["row_ptr"], op["col"], op["w"], op["kappa"], op["s"], dtype=dtype)
        Q2 = st["Q"].contiguous()
        lb.rk_step(plan2, Q2, st["dt"], 20 - st["step"], phys)
        assert torch.equal(Q2, ref)
        plan2.close()
