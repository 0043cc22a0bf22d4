"""The C ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(labfm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__ as g
    return g._builder().build()


def test_library_exports_every_declared_symbol(built_lib):
    declared = _declared_functions()
    assert "labfm_build_stencils" in declared and "labfm_rk_step" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(labfm_\w+)\b", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_the_header(built_lib):
    import paper_2102_02019_gb300 as lb
    assert lb.lib.labfm_abi_version() == 5
    assert lb.lib.labfm_last_error() == b""
    declared = set(_declared_functions())
    assert declared <= set(lb.exported_symbols()), declared - set(lb.exported_symbols())


def test_errors_are_reported_without_a_gpu(built_lib):
    import ctypes
    import paper_2102_02019_gb300 as lb
    # argument validation happens on the host before any CUDA call
    nnz = ctypes.c_int64(0)
    rc = lb.lib.labfm_build_stencils(None, None, 10, 1.0, 1.0, 3, None, None, 0, ctypes.byref(nnz), None)
    assert rc == 1 and b"null" in lb.lib.labfm_last_error()
    rc = lb.lib.labfm_build_weights(1, 1, 1, 10, 1.0, 1.0, 3, 1, 1, 10, 5, 1, 1, None, 1, None, None)
    assert rc == 1 and b"order m" in lb.lib.labfm_last_error()
    rc = lb.lib.labfm_rhs(None, 1, 2, None, None)
    assert rc == 1


def test_later_entry_points_validate_on_the_host(built_lib):
    import ctypes
    import paper_2102_02019_gb300 as lb
    L = lb.lib
    err = lambda: L.labfm_last_error()
    # stencil optimisation: order and shrink factor are checked before any launch
    assert L.labfm_stencil_optimise(1, 1, 1, 10, 1.0, 1.0, 3, 1, 1, 5, 0.99, 1.01, 1e-4, 10, 1, None, None, None) == 1
    assert b"order m" in err()
    assert L.labfm_stencil_optimise(1, 1, 1, 10, 1.0, 1.0, 3, 1, 1, 4, 1.0, 1.01, 1e-4, 10, 1, None, None, None) == 1
    assert b"factor" in err()
    assert L.labfm_stencil_optimise(1, 1, 1, 10, 1.0, 1.0, 3, 1, 1, 4, 0.99, 1.01, 0.0, 10, 1, None, None, None) == 1
    assert b"resid_coef" in err()
    assert L.labfm_modal_response(1, 1, 10, 1.0, 1.0, 3, 1, 1, 10, 1, 0, 1, None) == 1
    assert b"nk" in err()
    # plan-level calls on a null plan
    for fn, args in (("labfm_plan_set_staging", (None, 3, None)),
                     ("labfm_plan_set_persistent", (None, 1)),
                     ("labfm_plan_set_prefetch", (None, 2)),
                     ("labfm_rk_step_adjoint_recorded", (None, 1, 1, 1e-3, None, 1, 16, None))):
        assert getattr(L, fn)(*args) == 1, fn
    st = ctypes.c_int(0)
    assert L.labfm_plan_device_status(None, ctypes.byref(st)) == 1
    assert L.labfm_stage_states_bytes(None) == 0
    # objectives: null pointers and bad sizes
    out = ctypes.c_double(0.0)
    assert L.labfm_probe_momentum(None, 1, 1, 10, 0, ctypes.byref(out), None) == 1
    assert L.labfm_probe_momentum_grad(1, 1, 1, 0, 0, 1.0, 1, None) == 1
    assert b"N must be positive" in err()


def test_empty_and_oversize_inputs_are_rejected_on_the_host(built_lib):
    # N = 0 (an empty node set) and N >= 2^31 - 1 (beyond the int32 row pointers)
    # are EINVAL before any device access; the pointers are never dereferenced
    import ctypes
    import paper_2102_02019_gb300 as lb
    L = lb.lib
    p = 16  # non-null, never read
    nnz = ctypes.c_int64(-1)
    for N in (0, -3, 2 ** 31 - 1):
        assert L.labfm_build_stencils(p, p, N, 1.0, 1.0, 3, p, p, 0, ctypes.byref(nnz), None) == 1
        assert b"N out of range" in L.labfm_last_error()
        assert L.labfm_build_weights(p, p, p, N, 1.0, 1.0, 3, p, p, 0, 4, p, p, None, p, None,
                                     None) == 1
        assert b"N out of range" in L.labfm_last_error()
        plan = ctypes.c_void_p(1)
        assert L.labfm_plan_create(ctypes.byref(plan), N, 0, 1, p, None, p, p, p, None) == 1
        assert b"N out of range" in L.labfm_last_error() and plan.value is None
    assert nnz.value == -1


def test_binding_rejects_states_that_do_not_match_the_plan(built_lib):
    # the C entry points see only pointers, so a state of another element type or
    # with fewer than 3 N values would be read and written past its end: the
    # binding checks both before any launch (no GPU needed to see the refusal)
    import types

    import torch

    import paper_2102_02019_gb300 as lb
    plan = types.SimpleNamespace(N=10, dtype=torch.float64, handle=None, device="cpu")
    phys = lb.Phys(100.0, 0.005)
    s = torch.ones(10, dtype=torch.float64)
    calls = {
        "rk_step": lambda q: lb.rk_step(plan, q, 1e-3, 1, phys),
        "rk_step_noalloc": lambda q: lb.rk_step_noalloc(plan, q, 1e-3, 1, phys),
        "rhs": lambda q: lb.rhs(plan, q, phys),
        "filter": lambda q: lb.filter(plan, q),
        "stable_dt": lambda q: lb.stable_dt(plan, q, s, 10.0, 0.005),
        "rk_step_host": lambda q: lb.rk_step_host(plan, q, q, 1e-3, 1, phys),
        "rhs_adjoint": lambda q: lb.rhs_adjoint(plan, q, q, phys),
        "rk_step_adjoint": lambda q: lb.rk_step_adjoint(plan, q, q, 1e-3, phys),
        "rk_step_record": lambda q: lb.rk_step_record(plan, q, None, 1e-3, phys),
        "filter_adjoint": lambda q: lb.filter_adjoint(plan, q),
    }
    bad = {"float32": torch.zeros(3, 10, dtype=torch.float32),
           "short": torch.zeros(3, 9, dtype=torch.float64),
           "flat": torch.zeros(30, dtype=torch.float64)}
    for name, call in calls.items():
        for kind, q in bad.items():
            with pytest.raises(ValueError, match="plan|Q_host"):
                call(q)
    # a state that matches passes the check and is then refused for living on the host
    with pytest.raises(ValueError, match="CUDA"):
        lb.rk_step(plan, torch.zeros(3, 10, dtype=torch.float64), 1e-3, 1, phys)
    with pytest.raises(ValueError, match="float64 values"):
        lb.stable_dt(plan, torch.zeros(3, 10, dtype=torch.float64), s[:5], 10.0, 0.005)


def test_binding_rejects_node_sets_and_operators_of_the_wrong_shape(built_lib):
    # node sets, CSRs, weights and objective inputs outside a plan are checked for
    # element type and shape before any pointer is taken (CPU tensors: a tensor that
    # passed the checks would be refused next for living on the host)
    import torch

    import paper_2102_02019_gb300 as lb
    N = 8
    f64 = lambda *s: torch.zeros(*s, dtype=torch.float64)
    xy, h, s = f64(N, 2), f64(N), f64(N)
    rp = torch.zeros(N + 1, dtype=torch.int32)
    col = torch.zeros(16, dtype=torch.int32)
    w, kap = f64(6, 16), f64(N)
    calls = [
        (lambda: lb.build_stencils(xy.float(), h, 1.0, 1.0), "xy"),
        (lambda: lb.build_stencils(xy, h[:-1], 1.0, 1.0), "h"),
        (lambda: lb.build_weights(xy, h, s.float(), 1.0, 1.0, rp, col, 4), "s"),
        (lambda: lb.build_weights(xy, h, s, 1.0, 1.0, rp.long(), col, 4), "row_ptr"),
        (lambda: lb.build_weights(xy, h, s, 1.0, 1.0, rp[:-1], col, 4), "row_ptr"),
        (lambda: lb.build_weights(xy, h, s, 1.0, 1.0, rp, col.long(), 4), "col"),
        (lambda: lb.weight_coefficients(xy.T.contiguous(), h, s, 1.0, 1.0, rp, col, 4), "xy"),
        (lambda: lb.stencil_optimise(xy, h, s[:3], 1.0, 1.0, rp, col, 4), "s"),
        (lambda: lb.modal_response(xy, s, 1.0, 1.0, rp, col, w[:5]), "w"),
        (lambda: lb.modal_response(xy, s, 1.0, 1.0, rp, col, w.float()), "w"),
        (lambda: lb.build_wall_operator(xy, h, s.float(), 1.0, 1.0, 6, 4, torch.zeros(1, 5, dtype=torch.int32),
                                        f64(1, 2)), "s"),
        (lambda: lb.rhs_matrix_free(xy, h, 1.0, 1.0, rp, col, 4, f64(N * 90), f64(3, N), lb.Phys(1.0, 0.0),
                                    out=torch.zeros(3, N)), "out"),
        (lambda: lb.Plan(rp, col, w.float(), kap, s), "w"),
        (lambda: lb.Plan(rp, col, w[:, :8], kap, s), "w"),
        (lambda: lb.Plan(rp, col, w, kap[:4], s), "kappa"),
        (lambda: lb.Plan(rp, col.long(), w, kap, s), "col"),
        (lambda: lb.Plan.batched([dict(row_ptr=rp, col=col, w=w, kappa=kap, s=s.float())]), "instance 0: s"),
        (lambda: lb.kinetic_energy(f64(3, N), s[:4]), "s"),
        (lambda: lb.kinetic_energy(f64(2, N), s), "q"),
        (lambda: lb.probe_momentum(f64(3, N), s.float(), s), "px"),
        (lambda: lb.probe_momentum_grad(torch.zeros(3, N), s, s[:2]), "py"),
        (lambda: lb.conserved_vjp(f64(3, N), torch.zeros(3, N)), "qbar"),
        (lambda: lb.conserved_to_primitive(torch.zeros(3, N, dtype=torch.int32)), "c"),
    ]
    for call, name in calls:
        with pytest.raises(ValueError, match=name):
            call()
    # well-formed arguments pass the checks and are refused for living on the host
    with pytest.raises(ValueError, match="CUDA"):
        lb.build_weights(xy, h, s, 1.0, 1.0, rp, col, 4)
    with pytest.raises(ValueError, match="CUDA"):
        lb.Plan(rp, col, w, kap, s)
