"""Failure detection on the host: LABFM_FAULT makes the library's entry points
fail as they would on a real fault, before they touch the device, so that a
caller's error handling can be tested without a GPU and without faulting one."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g._builder().build()
    import paper_2102_02019_gb300 as lb
    return lb.lib


P = 16  # a non-null pointer that the injected paths never dereference


def test_alloc_fault_fails_every_allocating_entry_point_on_the_host(L, monkeypatch):
    monkeypatch.setenv("LABFM_FAULT", "alloc")
    plan = ctypes.c_void_p(1)
    assert L.labfm_plan_create(ctypes.byref(plan), 10, 0, 1, P, None, P, P, P, None) == 3
    assert b"injected" in L.labfm_last_error() and plan.value is None
    n = ctypes.c_int64(1)
    arr = (ctypes.c_int64 * 1)(10)
    nz = (ctypes.c_int64 * 1)(0)
    ptrs = (ctypes.c_void_p * 1)(P)
    assert L.labfm_plan_create_batched(ctypes.byref(plan), 1, ctypes.cast(arr, ctypes.c_void_p),
                                       ctypes.cast(nz, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                                       ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                                       ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                                       1, None) == 3
    assert b"labfm_plan_create_batched" in L.labfm_last_error()
    assert L.labfm_build_stencils(P, P, 10, 1.0, 1.0, 3, P, P, 100, ctypes.byref(n), None) == 3
    assert b"labfm_build_stencils" in L.labfm_last_error() and n.value == 1
    assert L.labfm_build_weights(P, P, P, 10, 1.0, 1.0, 3, P, P, 10, 4, P, P, None, P, ctypes.byref(n),
                                 None) == 3
    # argument errors still come first
    assert L.labfm_plan_create(ctypes.byref(plan), 0, 0, 1, P, None, P, P, P, None) == 1


def test_capacity_fault_reports_the_size_it_would_need(L, monkeypatch):
    monkeypatch.setenv("LABFM_FAULT", "capacity")
    n = ctypes.c_int64(-1)
    assert L.labfm_build_stencils(P, P, 10, 1.0, 1.0, 3, P, P, 250, ctypes.byref(n), None) == 4
    assert n.value == 251 and b"injected" in L.labfm_last_error()
    # the allocation paths are not affected by a capacity fault
    plan = ctypes.c_void_p(1)
    assert L.labfm_plan_create(ctypes.byref(plan), 0, 0, 1, P, None, P, P, P, None) == 1


def test_no_fault_without_a_recognised_setting(L, monkeypatch):
    # argument validation alone decides these calls: nothing is injected for an
    # unset variable or an unknown value
    for value in (None, "", "bogus", "singular_node:", "singular_node:x"):
        if value is None:
            monkeypatch.delenv("LABFM_FAULT", raising=False)
        else:
            monkeypatch.setenv("LABFM_FAULT", value)
        n = ctypes.c_int64(-1)
        assert L.labfm_build_stencils(P, P, 0, 1.0, 1.0, 3, P, P, 0, ctypes.byref(n), None) == 1
        assert b"N out of range" in L.labfm_last_error()
