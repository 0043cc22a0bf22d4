"""Python binding of liblabfm (the GB300 LABFM hot path).

Argument marshalling only: every step runs in the CUDA kernels of liblabfm.so,
reached through its C ABI (include/labfm.h) with ctypes.  PyTorch supplies
device memory and the current CUDA stream.  There is no CPU fallback: if the
library is missing or fails to load, importing the binding raises.

Functions keep the names of the C entry points:

    build_stencils(xy, h, Lx, Ly)        -> (row_ptr, col)
    build_weights(xy, h, s, Lx, Ly, row_ptr, col, m) -> dict(w, kappa, status, residual)
    Plan(N, row_ptr, col, w, kappa, s, dtype)  (labfm_plan_create / _destroy)
    rhs(plan, fields, phys)              -> 3 x N
    filter(plan, fields)                 -> 3 x N
    rk_step(plan, Q, dt, nsteps, phys)   (in place)
    stable_dt(plan, fields, s, c, mu)    -> 1-element device tensor
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblabfm.so")

LABFM_F64 = 0
LABFM_F32 = 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "ECAPACITY",
                5: "ESINGULAR", 6: "ENONFINITE", 7: "ETIMEOUT"}
NODE_FEW_NEIGHBOURS = 1
NODE_SINGULAR = 2
NODE_NONFINITE = 4
OPS = ("x", "y", "xx", "xy", "yy", "hyp")


class LabfmError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class _Phys(ctypes.Structure):
    _fields_ = [("c2", ctypes.c_double), ("mu", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double)]


class _Nscbc(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("L", ctypes.c_double), ("mach", ctypes.c_double),
                ("rho0", ctypes.c_double)]


WALL, INFLOW, OUTFLOW = 0, 1, 2


class _PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nnz_padded", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("group", ctypes.c_int32), ("block", ctypes.c_int32),
                ("n_instances", ctypes.c_int32), ("entry_bytes", ctypes.c_int32),
                ("filter_entry_bytes", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("prefetch", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("filter_group", ctypes.c_int32), ("filter_persistent", ctypes.c_int32),
                ("programmatic", ctypes.c_int32)]


class _Profile(ctypes.Structure):
    _fields_ = [("stage_ms", ctypes.c_double), ("stage_launches", ctypes.c_int64),
                ("filter_ms", ctypes.c_double), ("filter_launches", ctypes.c_int64),
                ("dropped", ctypes.c_int64),
                ("rec_stage_ms", ctypes.c_double), ("rec_stage_launches", ctypes.c_int64),
                ("adj_a_ms", ctypes.c_double), ("adj_a_launches", ctypes.c_int64),
                ("adj_b_ms", ctypes.c_double), ("adj_b_launches", ctypes.c_int64),
                ("adj_filter_ms", ctypes.c_double), ("adj_filter_launches", ctypes.c_int64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "labfm_last_error": (ctypes.c_char_p, []),
    "labfm_abi_version": (_I32, []),
    "labfm_build_stencils": (_I32, [_P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I64,
                                    ctypes.POINTER(_I64), _P]),
    "labfm_build_weights": (_I32, [_P, _P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I64, _I32,
                                   _P, _P, _P, _P, ctypes.POINTER(_I64), _P]),
    "labfm_stencil_optimise": (_I32, [_P, _P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I32, _D, _D,
                                      _D, _I32, _P, _P, _P, _P]),
    "labfm_modal_response": (_I32, [_P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I64, _P, _I32, _P,
                                    _P]),
    "labfm_build_wall_operator": (_I32, [_P, _P, _P, _I64, _D, _D, ctypes.c_uint32, _I32, _I32, _I64, _P, _P,
                                         _D, _P, _P, _I64, ctypes.POINTER(_I64), _P, _P, _P,
                                         ctypes.POINTER(_I64), _P]),
    "labfm_plan_set_walls": (_I32, [_P, _I64, _P, _P, _P]),
    "labfm_build_weights_ex": (_I32, [_P, _P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I64, _I32,
                                      _P, _P, _P, _P, ctypes.POINTER(_I64), _P, _P]),
    "labfm_weight_coefficients_per_node": (ctypes.c_size_t, [_I32]),
    "labfm_rhs_matrix_free": (_I32, [_P, _P, _I64, _D, _D, ctypes.c_uint32, _P, _P, _I32, _P, _P, _P,
                                     ctypes.POINTER(_Phys), _P]),
    "labfm_plan_set_boundaries": (_I32, [_P, _I64, _P, _P, _P, _P, ctypes.POINTER(_Nscbc), _P]),
    "labfm_plan_create": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I32, _P, _P, _P, _P, _P, _P]),
    "labfm_plan_destroy": (_I32, [_P]),
    "labfm_plan_get_info": (_I32, [_P, ctypes.POINTER(_PlanInfo)]),
    "labfm_plan_set_launch": (_I32, [_P, _I32, _I32]),
    "labfm_plan_set_filter_launch": (_I32, [_P, _I32, _I32]),
    "labfm_plan_set_launch_ranges": (_I32, [_P, _I32, _P, _P, _P]),
    "labfm_plan_autotune": (_I32, [_P, _P, _P, ctypes.POINTER(_Phys), _I32,
                                   ctypes.POINTER(_I32), ctypes.POINTER(_I32), _P]),
    "labfm_rhs": (_I32, [_P, _P, _P, ctypes.POINTER(_Phys), _P]),
    "labfm_filter": (_I32, [_P, _P, _P, _P]),
    "labfm_rk_workspace_bytes": (ctypes.c_size_t, [_P]),
    "labfm_rk_step": (_I32, [_P, _P, _P, ctypes.c_size_t, _D, _I32, ctypes.POINTER(_Phys), _P]),
    "labfm_stable_dt": (_I32, [_P, _P, _P, _D, _D, _P, _P]),
    "labfm_rk_step_host": (_I32, [_P, _P, _P, _P, ctypes.c_size_t, _D, _I32, ctypes.POINTER(_Phys), _P]),
    "labfm_plan_set_profiling": (_I32, [_P, _I32]),
    "labfm_plan_read_profile": (_I32, [_P, ctypes.POINTER(_Profile)]),
    "labfm_probe_fma_rate": (_I32, [_I32, ctypes.POINTER(_D)]),
    "labfm_rk_step_noalloc": (_I32, [_P, _P, _D, _I32, ctypes.POINTER(_Phys), _P]),
    "labfm_plan_create_batched": (_I32, [ctypes.POINTER(_P), _I32, _P, _P, _P, _P, _P, _P, _P, _I32, _P]),
    "labfm_plan_set_dt": (_I32, [_P, _P, _P]),
    "labfm_stable_dt_instances": (_I32, [_P, _P, _P, _D, _D, _P, _P]),
    "labfm_plan_set_persistent": (_I32, [_P, _I32]),
    "labfm_plan_set_prefetch": (_I32, [_P, _I32]),
    "labfm_plan_set_programmatic_launch": (_I32, [_P, _I32]),
    "labfm_plan_set_staging": (_I32, [_P, _I32, _P]),
    "labfm_plan_device_status": (_I32, [_P, ctypes.POINTER(_I32)]),
    "labfm_plan_set_wait_limit": (_I32, [_P, _I64]),
    "labfm_plan_set_check_finite": (_I32, [_P, _I32]),
    "labfm_step_graph_create": (_I32, [ctypes.POINTER(_P), _P, _P, ctypes.c_size_t, _D, ctypes.POINTER(_Phys)]),
    "labfm_step_graph_run": (_I32, [_P, _P, _I32, _P]),
    "labfm_step_graph_destroy": (_I32, [_P]),
    "labfm_plan_enable_adjoint": (_I32, [_P, _P]),
    "labfm_adjoint_workspace_bytes": (ctypes.c_size_t, [_P]),
    "labfm_rhs_adjoint": (_I32, [_P, _P, _P, _P, ctypes.POINTER(_Phys), _P, ctypes.c_size_t, _P]),
    "labfm_rk_step_adjoint": (_I32, [_P, _P, _P, _D, ctypes.POINTER(_Phys), _P, ctypes.c_size_t, _P]),
    "labfm_filter_adjoint": (_I32, [_P, _P, _P, _P, ctypes.c_size_t, _P]),
    "labfm_stage_states_bytes": (ctypes.c_size_t, [_P]),
    "labfm_rk_step_record": (_I32, [_P, _P, _P, ctypes.c_size_t, _P, ctypes.c_size_t, _D,
                                    ctypes.POINTER(_Phys), _P]),
    "labfm_rk_step_adjoint_recorded": (_I32, [_P, _P, _P, _D, ctypes.POINTER(_Phys), _P, ctypes.c_size_t,
                                              _P]),
    "labfm_conserved_to_primitive": (_I32, [_P, _P, _I64, _I32, _P]),
    "labfm_conserved_vjp": (_I32, [_P, _P, _P, _I64, _I32, _P]),
    "labfm_kinetic_energy": (_I32, [_P, _P, _I64, _I32, _P, _P]),
    "labfm_kinetic_energy_grad": (_I32, [_P, _P, _I64, _I32, _D, _P, _P]),
    "labfm_probe_momentum": (_I32, [_P, _P, _P, _I64, _I32, _P, _P]),
    "labfm_probe_momentum_grad": (_I32, [_P, _P, _P, _I64, _I32, _D, _P, _P]),
}


# the C ABI this binding's signatures and structures follow (include/labfm.h)
ABI_VERSION = 5


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
            "(needs nvcc).  There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.labfm_abi_version() != ABI_VERSION:
        raise ImportError(f"{LIB_PATH} has ABI {lib.labfm_abi_version()}, this binding needs "
                          f"{ABI_VERSION}: rebuild it (`__graft_entry__.build()`)")
    return lib


lib = _load()


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def _check(rc: int) -> None:
    if rc != 0:
        raise LabfmError(rc, lib.labfm_last_error().decode())


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("liblabfm takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("liblabfm takes contiguous tensors")
    return t.data_ptr()


def _state(plan, t: torch.Tensor, name: str = "Q") -> int:
    """Device pointer of a 3 x N state of the plan's element type.  The C side sees
    only a pointer, so a tensor of another dtype or fewer than 3 N elements would
    make the kernels read and write past its end: both are checked here, before
    any launch."""
    if t.dtype != plan.dtype:
        raise ValueError(f"{name} is {t.dtype} but the plan computes in {plan.dtype}")
    if tuple(t.shape) != (3, plan.N):
        raise ValueError(f"{name} has shape {tuple(t.shape)}; the plan needs (3, {plan.N})")
    return _ptr(t)


def _nodes(plan, t: torch.Tensor, name: str) -> torch.Tensor:
    """N float64 node values (node spacing s), checked like _state; returns t."""
    if t.dtype != torch.float64 or t.numel() != plan.N:
        raise ValueError(f"{name} must hold {plan.N} float64 values")
    return t


# Argument checks of the calls that take node sets, operators and states outside a
# plan.  The C side sees only pointers and counts derived from the shapes, so a
# tensor of another element type or of fewer elements would be read (or written)
# past its end; each check runs before the tensor's pointer is taken.

def _check_tensor(t: torch.Tensor, dtype: torch.dtype, shape: tuple, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be {dtype} of shape {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    return t


def _node_set(xy: torch.Tensor, **per_node) -> int:
    """N of an (N, 2) float64 position tensor; every keyword tensor must hold N float64
    values (None is skipped)."""
    if not isinstance(xy, torch.Tensor) or xy.dim() != 2 or xy.shape[1] != 2 or xy.dtype != torch.float64:
        raise ValueError("xy must be float64 of shape (N, 2)")
    N = int(xy.shape[0])
    for name, t in per_node.items():
        if t is not None:
            _check_tensor(t, torch.float64, (N,), name)
    return N


def _csr(row_ptr: torch.Tensor, col: torch.Tensor, N: int) -> None:
    """int32 row pointers (N + 1) and columns (one dimension)."""
    _check_tensor(row_ptr, torch.int32, (N + 1,), "row_ptr")
    if not isinstance(col, torch.Tensor) or col.dtype != torch.int32 or col.dim() != 1:
        raise ValueError("col must be a one-dimensional int32 tensor")


def _field_dtype(t: torch.Tensor, name: str, rows: int = 3) -> int:
    """N of a (rows, N) float32 or float64 tensor."""
    if not isinstance(t, torch.Tensor) or t.dtype not in (torch.float32, torch.float64) or t.dim() != 2 \
            or t.shape[0] != rows:
        raise ValueError(f"{name} must be float32 or float64 of shape ({rows}, N)")
    return int(t.shape[1])


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class Phys:
    """c2 = c^2, mu, body force (gx, gy) of eq. icns."""
    c2: float
    mu: float
    gx: float = 0.0
    gy: float = 0.0

    def c(self) -> _Phys:
        return _Phys(self.c2, self.mu, self.gx, self.gy)


def build_stencils(xy: torch.Tensor, h: torch.Tensor, Lx: float, Ly: float,
                   periodic=(True, True), stream=None):
    """CSR (row_ptr int32 [N+1], col int32 [nnz]) of |r_ji| <= 2 h_i (labfm_build_stencils)."""
    N = _node_set(xy, h=h)
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    row_ptr = torch.empty(N + 1, dtype=torch.int32, device=xy.device)
    nnz = _I64(0)
    st = _stream(stream)
    _check(lib.labfm_build_stencils(_ptr(xy), _ptr(h), N, Lx, Ly, mask, _ptr(row_ptr), None, 0,
                                    ctypes.byref(nnz), st))
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=xy.device)
    _check(lib.labfm_build_stencils(_ptr(xy), _ptr(h), N, Lx, Ly, mask, _ptr(row_ptr), _ptr(col),
                                    col.numel(), ctypes.byref(nnz), st))
    return row_ptr, col[:nnz.value]


def build_weights(xy, h, s, Lx, Ly, row_ptr, col, m, periodic=(True, True), residual=True,
                  check=False, stream=None):
    """FP64 weights (labfm_build_weights): dict with w (6, nnz), kappa, status, residual, n_failed.

    With check=True the call synchronises and raises LabfmError(ESINGULAR) if a node failed."""
    N = _node_set(xy, h=h, s=s)
    _csr(row_ptr, col, N)
    nnz = col.numel()
    dev = xy.device
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    w = torch.empty((6, max(nnz, 1)), dtype=torch.float64, device=dev)
    kappa = torch.empty(N, dtype=torch.float64, device=dev)
    status = torch.empty(N, dtype=torch.int32, device=dev)
    res = torch.empty(N, dtype=torch.float64, device=dev) if residual else None
    nf = _I64(0)
    rc = lib.labfm_build_weights(_ptr(xy), _ptr(h), _ptr(s), N, Lx, Ly, mask, _ptr(row_ptr),
                                 _ptr(col) if nnz else None, nnz, m, _ptr(w), _ptr(kappa), _ptr(res),
                                 _ptr(status), ctypes.byref(nf) if check else None, _stream(stream))
    _check(rc)
    return {"w": w[:, :nnz] if nnz else w[:, :0], "kappa": kappa, "status": status,
            "residual": res, "n_failed": nf.value if check else None}


def weight_coefficients(xy, h, s, Lx, Ly, row_ptr, col, m, periodic=(True, True), weights=False,
                        check=False, stream=None):
    """labfm_build_weights_ex: every node's weight polynomials (N, (m+1)(m+2)/2, 6) for the
    matrix-free right-hand side, with kappa and status; weights=True also returns the
    stored weights w (6, nnz)."""
    N = _node_set(xy, h=h, s=s)
    _csr(row_ptr, col, N)
    nnz = col.numel()
    dev = xy.device
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    nc = int(lib.labfm_weight_coefficients_per_node(int(m)))
    if nc == 0:
        raise ValueError("order m must be even and in [2, 10]")
    coef = torch.empty((N, nc // 6, 6), dtype=torch.float64, device=dev)
    w = torch.empty((6, max(nnz, 1)), dtype=torch.float64, device=dev) if weights else None
    kappa = torch.empty(N, dtype=torch.float64, device=dev)
    status = torch.empty(N, dtype=torch.int32, device=dev)
    nf = _I64(0)
    _check(lib.labfm_build_weights_ex(_ptr(xy), _ptr(h), _ptr(s), N, Lx, Ly, mask, _ptr(row_ptr),
                                      _ptr(col) if nnz else None, nnz, m, _ptr(w), _ptr(kappa), None,
                                      _ptr(status), ctypes.byref(nf) if check else None, _ptr(coef),
                                      _stream(stream)))
    out = {"coef": coef, "kappa": kappa, "status": status, "n_failed": nf.value if check else None}
    if weights:
        out["w"] = w[:, :nnz]
    return out


def rhs_matrix_free(xy, h, Lx, Ly, row_ptr, col, m, coef, fields, phys, periodic=(True, True),
                    out=None, stream=None):
    """labfm_rhs_matrix_free: the FP64 eq. icns right-hand side with every neighbour's
    weights recomputed from the weight polynomials (3 x N float64)."""
    N = _node_set(xy, h=h)
    _csr(row_ptr, col, N)
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    if fields.dtype != torch.float64 or fields.numel() < 3 * N or not fields.is_contiguous():
        raise ValueError("fields must be a contiguous float64 tensor of 3 x N values")
    if coef.dtype != torch.float64 or coef.numel() < N * int(lib.labfm_weight_coefficients_per_node(int(m))):
        raise ValueError("coef must be the float64 weight polynomials of order m")
    out = torch.empty_like(fields) if out is None else out
    if out.dtype != torch.float64 or out.numel() < 3 * N:
        raise ValueError("out must be a float64 tensor of 3 x N values")
    ph = phys.c()
    _check(lib.labfm_rhs_matrix_free(_ptr(xy), _ptr(h), N, Lx, Ly, mask, _ptr(row_ptr),
                                     _ptr(col) if col.numel() else None, int(m), _ptr(coef), _ptr(fields),
                                     _ptr(out), ctypes.byref(ph), _stream(stream)))
    return out


def stencil_optimise(xy, h0, s, Lx, Ly, row_ptr, col, m, factor=0.99, amp_max=1.01, resid_coef=1e-4,
                     max_iter=400, periodic=(True, True), alpha=False, stream=None):
    """labfm_stencil_optimise: per-node optimised h (Section 4) and the number of systems
    solved per node, as (h, solves) device tensors, and with alpha=True also the
    (N, 2) Laplacian residuals alpha_L at the returned h and where the iteration
    stopped.  resid_coef=math.inf switches the Laplacian-residual test off."""
    N = _node_set(xy, h0=h0, s=s)
    _csr(row_ptr, col, N)
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    h = torch.empty(N, dtype=torch.float64, device=xy.device)
    solves = torch.empty(N, dtype=torch.int32, device=xy.device)
    al = torch.empty((N, 2), dtype=torch.float64, device=xy.device) if alpha else None
    _check(lib.labfm_stencil_optimise(_ptr(xy), _ptr(h0), _ptr(s), N, Lx, Ly, mask, _ptr(row_ptr),
                                      _ptr(col), m, factor, amp_max, resid_coef, max_iter, _ptr(h), _ptr(solves),
                                      _ptr(al), _stream(stream)))
    return (h, solves, al) if alpha else (h, solves)


def build_wall_operator(xy, h, s, Lx, Ly, m, m_wall, wall_column, wall_normal, h1d_over_s=1.7,
                        periodic=(True, False), check=False, stream=None):
    """labfm_build_wall_operator (Section 7.1): the operator of a domain with walls as
    dict(row_ptr, col, w (6, nnz), kappa, status, n_failed), ready for Plan.
    wall_column: (n_wall, 5) int32 nodes q = 0..4 of each wall column; wall_normal:
    (n_wall, 2) float64 inward unit normals."""
    N = _node_set(xy, h=h, s=s)
    n_wall = wall_column.shape[0]
    if wall_column.dtype != torch.int32 or tuple(wall_column.shape) != (n_wall, 5):
        raise ValueError("wall_column must be int32 of shape (n_wall, 5)")
    if wall_normal.dtype != torch.float64 or tuple(wall_normal.shape) != (n_wall, 2):
        raise ValueError("wall_normal must be float64 of shape (n_wall, 2)")
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    row_ptr = torch.empty(N + 1, dtype=torch.int32, device=xy.device)
    nnz = _I64(0)
    st = _stream(stream)
    args = (_ptr(xy), _ptr(h), _ptr(s), N, Lx, Ly, mask, m, m_wall, n_wall, _ptr(wall_column),
            _ptr(wall_normal), float(h1d_over_s), _ptr(row_ptr))
    _check(lib.labfm_build_wall_operator(*args, None, 0, ctypes.byref(nnz), None, None, None, None, st))
    n = nnz.value
    col = torch.empty(max(n, 1), dtype=torch.int32, device=xy.device)
    w = torch.empty((6, max(n, 1)), dtype=torch.float64, device=xy.device)
    kappa = torch.empty(N, dtype=torch.float64, device=xy.device)
    status = torch.empty(N, dtype=torch.int32, device=xy.device)
    nf = _I64(0)
    _check(lib.labfm_build_wall_operator(*args, _ptr(col), col.numel(), ctypes.byref(nnz), _ptr(w),
                                         _ptr(kappa), _ptr(status), ctypes.byref(nf) if check else None, st))
    return {"row_ptr": row_ptr, "col": col[:n], "w": w[:, :n], "kappa": kappa, "status": status,
            "n_failed": nf.value if check else None}


def modal_response(xy, s, Lx, Ly, row_ptr, col, w, nk=16, periodic=(True, True), stream=None):
    """labfm_modal_response: (N, 3, nk) amplitude responses of d/dx, d/dy and the
    Laplacian of FP64 weights w (6, nnz) (Section 3)."""
    N = _node_set(xy, s=s)
    _csr(row_ptr, col, N)
    nnz = col.numel()
    _check_tensor(w, torch.float64, (6, nnz), "w")
    mask = (1 if periodic[0] else 0) | (2 if periodic[1] else 0)
    w = w.contiguous()
    out = torch.empty((N, 3, nk), dtype=torch.float64, device=xy.device)
    _check(lib.labfm_modal_response(_ptr(xy), _ptr(s), N, Lx, Ly, mask, _ptr(row_ptr),
                                    _ptr(col) if nnz else None, nnz, _ptr(w), nk, _ptr(out),
                                    _stream(stream)))
    return out


class Plan:
    """A prepared operator for the step kernels (labfm_plan_create / labfm_plan_destroy)."""

    @classmethod
    def batched(cls, instances, dtype=torch.float32, stream=None):
        """labfm_plan_create_batched over a list of dicts with row_ptr, col, w, kappa, s."""
        n = len(instances)
        for k, d in enumerate(instances):
            cls._check_operator(d["row_ptr"], d["col"], d["w"], d["kappa"], d["s"], where=f"instance {k}: ")
        arr = lambda vals, ct: (ct * n)(*vals)
        Ns = arr([d["row_ptr"].numel() - 1 for d in instances], _I64)
        nnzs = arr([d["col"].numel() for d in instances], _I64)
        ptrs = {k: arr([_ptr(d[k]) if d[k].numel() else None for d in instances], _P)
                for k in ("row_ptr", "col", "w", "kappa", "s")}
        self = cls.__new__(cls)
        self.N = int(sum(Ns))
        self.nnz = int(sum(nnzs))
        self.dtype = dtype
        self.device = instances[0]["row_ptr"].device
        self._keep = [d["w"].contiguous() for d in instances]
        handle = _P()
        _check(lib.labfm_plan_create_batched(
            ctypes.byref(handle), n, ctypes.cast(Ns, _P), ctypes.cast(nnzs, _P),
            ctypes.cast(ptrs["row_ptr"], _P), ctypes.cast(ptrs["col"], _P),
            ctypes.cast(ptrs["w"], _P), ctypes.cast(ptrs["kappa"], _P), ctypes.cast(ptrs["s"], _P),
            LABFM_F32 if dtype == torch.float32 else LABFM_F64, _stream(stream)))
        self._h = handle
        self.n_instances = n
        self.offsets = [0]
        for v in Ns:
            self.offsets.append(self.offsets[-1] + int(v))
        return self

    def set_dt(self, dt_inst, stream=None):
        """labfm_plan_set_dt: per-instance time steps (host sequence)."""
        vals = (_D * len(dt_inst))(*[float(v) for v in dt_inst])
        _check(lib.labfm_plan_set_dt(self._h, ctypes.cast(vals, _P), _stream(stream)))

    def stable_dt_instances(self, fields, s, c, mu, stream=None):
        """labfm_stable_dt_instances: eq. dt per instance (float64 device tensor)."""
        _nodes(self, s, "s")
        fp, sp = _state(self, fields, "fields"), _ptr(s)
        out = torch.empty(getattr(self, "n_instances", 1), dtype=torch.float64, device=fields.device)
        _check(lib.labfm_stable_dt_instances(self._h, fp, sp, float(c), float(mu),
                                             _ptr(out), _stream(stream)))
        return out

    def set_persistent(self, enable: bool = True) -> None:
        _check(lib.labfm_plan_set_persistent(self._h, 1 if enable else 0))

    def set_prefetch(self, distance: int) -> None:
        """labfm_plan_set_prefetch: L2 prefetch distance of the F32 record stream (0 = off)."""
        _check(lib.labfm_plan_set_prefetch(self._h, int(distance)))

    def set_programmatic_launch(self, enable: bool = True) -> None:
        """labfm_plan_set_programmatic_launch: programmatic dependent launches of the
        plan's kernels (on by default) or plain launches; results are the same."""
        _check(lib.labfm_plan_set_programmatic_launch(self._h, 1 if enable else 0))

    def set_staging(self, stages: int = 3, stream=None) -> None:
        """labfm_plan_set_staging: shared-memory staging of the operator stream for the
        F32 stage kernel with 16 or 32 lanes per node (0 = off)."""
        _check(lib.labfm_plan_set_staging(self._h, int(stages), _stream(stream)))

    def set_walls(self, wall_nodes: torch.Tensor, wall_normal: torch.Tensor, stream=None) -> None:
        """labfm_plan_set_walls: no-slip walls (Section 7.1) at the given nodes (int32,
        n_wall) with inward unit normals (float64, (n_wall, 2)); an empty wall_nodes
        removes them."""
        n = wall_nodes.numel()
        if wall_nodes.dtype != torch.int32 or (n and (wall_normal.dtype != torch.float64
                                                      or tuple(wall_normal.shape) != (n, 2))):
            raise ValueError("wall_nodes int32 (n_wall,), wall_normal float64 (n_wall, 2)")
        _check(lib.labfm_plan_set_walls(self._h, n, _ptr(wall_nodes) if n else None,
                                        _ptr(wall_normal.contiguous()) if n else None, _stream(stream)))

    def set_boundaries(self, nodes: torch.Tensor, normal: torch.Tensor, kind: torch.Tensor,
                       target: torch.Tensor, sigma: float = 0.278, L: float = 1.0, mach: float = 0.0,
                       rho0: float = 1.0, stream=None) -> None:
        """labfm_plan_set_boundaries: walls, inflows and outflows (Section 7.1).  nodes,
        kind: int32 (n,); normal, target: float64 (n, 2)."""
        n = nodes.numel()
        for t, dt_, shape, name in ((nodes, torch.int32, (n,), "nodes"), (kind, torch.int32, (n,), "kind"),
                                    (normal, torch.float64, (n, 2), "normal"),
                                    (target, torch.float64, (n, 2), "target")):
            if t.dtype != dt_ or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be {dt_} of shape {shape}")
        prm = _Nscbc(float(sigma), float(L), float(mach), float(rho0))
        args = [_ptr(t.contiguous()) if n else None for t in (nodes, normal, kind, target)]
        _check(lib.labfm_plan_set_boundaries(self._h, n, *args, ctypes.byref(prm), _stream(stream)))

    def set_wait_limit(self, limit_ns: int) -> None:
        """labfm_plan_set_wait_limit: limit of the staged kernel's bounded waits (ns;
        0 = one non-blocking test, which makes the waits run out)."""
        _check(lib.labfm_plan_set_wait_limit(self._h, int(limit_ns)))

    def set_check_finite(self, every: int) -> None:
        """labfm_plan_set_check_finite: check the state for non-finite values every
        `every` steps of rk_step (and after its last); 0 turns it off."""
        _check(lib.labfm_plan_set_check_finite(self._h, int(every)))

    def device_status(self) -> int:
        """labfm_plan_device_status: LABFM_OK (0), LABFM_ENONFINITE (6) or
        LABFM_ETIMEOUT (7); clears it."""
        st = _I32(0)
        _check(lib.labfm_plan_device_status(self._h, ctypes.byref(st)))
        return st.value

    def __init__(self, row_ptr, col, w, kappa, s, dtype=torch.float32, stream=None):
        self._check_operator(row_ptr, col, w, kappa, s)
        self.N = row_ptr.numel() - 1
        self.nnz = col.numel()
        self.dtype = dtype
        code = LABFM_F32 if dtype == torch.float32 else LABFM_F64
        if dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be float32 or float64")
        w = w.contiguous()
        handle = _P()
        _check(lib.labfm_plan_create(ctypes.byref(handle), self.N, self.nnz, code, _ptr(row_ptr),
                                     _ptr(col) if self.nnz else None, _ptr(w), _ptr(kappa), _ptr(s),
                                     _stream(stream)))
        self._h = handle
        self.device = row_ptr.device

    @staticmethod
    def _check_operator(row_ptr, col, w, kappa, s, where=""):
        if not isinstance(row_ptr, torch.Tensor) or row_ptr.dim() != 1 or row_ptr.numel() < 1:
            raise ValueError(f"{where}row_ptr must be a one-dimensional int32 tensor of N + 1 values")
        N = row_ptr.numel() - 1
        _csr(row_ptr, col, N)
        _check_tensor(w, torch.float64, (6, col.numel()), where + "w")
        _check_tensor(kappa, torch.float64, (N,), where + "kappa")
        _check_tensor(s, torch.float64, (N,), where + "s")

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = _PlanInfo()
        _check(lib.labfm_plan_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _PlanInfo._fields_}

    def set_launch(self, group: int, block: int) -> None:
        _check(lib.labfm_plan_set_launch(self._h, group, block))

    def set_launch_ranges(self, begin, group, prefetch) -> None:
        """labfm_plan_set_launch_ranges: per node range [begin[r], begin[r+1]) its own
        lanes per node and prefetch distance (host sequences; empty removes them)."""
        n = len(group)
        b = (_I64 * (n + 1))(*[int(v) for v in begin]) if n else None
        g = (_I32 * n)(*[int(v) for v in group]) if n else None
        pf = (_I32 * n)(*[int(v) for v in prefetch]) if n else None
        _check(lib.labfm_plan_set_launch_ranges(self._h, n, ctypes.cast(b, _P) if n else None,
                                                ctypes.cast(g, _P) if n else None,
                                                ctypes.cast(pf, _P) if n else None))

    def tune_ranges(self, Q: torch.Tensor, phys: Phys, dt: float, classes, steps: int = 3,
                    groups=(2, 4, 8, 16), prefetch=(0, 2), cache: bool = True) -> list[dict]:
        """Per-class launch shapes for a plan whose order classes occupy contiguous node
        ranges.  classes: (begin, end, m, mean neighbours) per range, covering [0, N).
        For each class in turn (the others at their current choice) time `steps` RK
        steps for every lanes-per-node group and prefetch distance and keep the
        fastest, then set the ranges.  With cache=True a choice is read from and
        written to a JSON file (LABFM_TUNE_CACHE, else ~/.cache/labfm/tune.json) keyed
        by GPU name, m, mean-neighbour bucket (steps of 8) and dtype, and a class found
        there is not timed.  Q is not modified.  Returns the per-class choices."""
        import json as _json
        _state(self, Q)
        dname = "f32" if self.dtype == torch.float32 else "f64"
        gpu = torch.cuda.get_device_name(self.device)
        keys = [f"{gpu}|m{int(m)}|nn{int(nn) // 8 * 8}|{dname}" for _, _, m, nn in classes]
        path = os.environ.get("LABFM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "labfm",
                                                                   "tune.json")
        stored = {}
        if cache and os.path.exists(path):
            try:
                stored = _json.load(open(path))
            except (OSError, ValueError):
                stored = {}
        pfs = tuple(prefetch) if self.dtype == torch.float32 else (0,)
        begin = [int(c[0]) for c in classes] + [int(classes[-1][1])]
        choice = [dict(stored[k]) if k in stored else {"group": 4, "prefetch": pfs[-1]} for k in keys]
        from_cache = [k in stored for k in keys]
        work = workspace(self)

        def timed():
            self.set_launch_ranges(begin, [c["group"] for c in choice], [c["prefetch"] for c in choice])
            Qs = Q.clone()
            rk_step(self, Qs, dt, 1, phys, work=work)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            rk_step(self, Qs, dt, steps, phys, work=work)
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / steps

        for r in range(len(classes)):
            if from_cache[r]:
                continue
            best = None
            for g in groups:
                for pf in pfs:
                    choice[r] = {"group": g, "prefetch": pf}
                    ms = timed()
                    if best is None or ms < best[0]:
                        best = (ms, g, pf)
            choice[r] = {"group": best[1], "prefetch": best[2]}
            stored[keys[r]] = choice[r]
        ms = timed()
        if cache and not all(from_cache):
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                with open(path, "w") as f:
                    _json.dump(stored, f, indent=1, sort_keys=True)
            except OSError:
                pass
        return [dict(c, m=int(cl[2]), mean_neighbours=float(cl[3]), nodes=int(cl[1] - cl[0]), key=k,
                     from_cache=fc, ms_per_step=ms) for c, cl, k, fc in zip(choice, classes, keys, from_cache)]

    def set_filter_launch(self, group: int = 0, persistent: bool = False) -> None:
        """labfm_plan_set_filter_launch: the filter's lanes per node (0 = the plan's
        group) and its persistent grid-stride grid."""
        _check(lib.labfm_plan_set_filter_launch(self._h, int(group), 1 if persistent else 0))

    def autotune(self, fields: torch.Tensor, phys: Phys, reps: int = 5, stream=None):
        _state(self, fields, "fields")
        out = torch.empty_like(fields)
        g, b = _I32(0), _I32(0)
        ph = phys.c()
        _check(lib.labfm_plan_autotune(self._h, _ptr(fields), _ptr(out), ctypes.byref(ph), reps,
                                       ctypes.byref(g), ctypes.byref(b), _stream(stream)))
        return g.value, b.value

    def set_profiling(self, enable: bool = True, every: int = 1) -> None:
        """labfm_plan_set_profiling: launch timing on (every `every`-th step of
        rk_step timed) or off."""
        _check(lib.labfm_plan_set_profiling(self._h, int(every) if enable else 0))

    def read_profile(self) -> dict:
        pr = _Profile()
        _check(lib.labfm_plan_read_profile(self._h, ctypes.byref(pr)))
        return {k: getattr(pr, k) for k, _ in _Profile._fields_}

    def tune_step(self, Q: torch.Tensor, phys: Phys, dt: float, steps: int = 3,
                  groups=(2, 4, 8, 16), staged=((16, 3), (32, 3), (32, 4)),
                  prefetch=(0, 2), filter_groups=(2, 4, 8, 16), filter_blocks=(64, 128)) -> dict:
        """Autotune the time step itself: time `steps` RK steps (CUDA events) for every
        lanes-per-node group with the plain and the persistent stage kernel (F32: with
        each L2 prefetch distance), and (F32) for the staged kernel at the given (lanes
        per node, ring slots), keep the fastest; then, with that stage kernel, time the
        filter's own lanes per node with its plain and persistent grids and the plan's
        block size (which only the filter and filter-transpose kernels use; the stage and
        adjoint gather kernels run one-warp blocks), and keep the fastest.  Q is not modified.  Returns the chosen configuration."""
        _state(self, Q)
        info = self.info()
        block = info["block"]
        pfs = tuple(prefetch) if self.dtype == torch.float32 else (info["prefetch"],)
        configs = [(g, p, 0, pf) for pf in pfs for p in (False, True) for g in groups]
        if self.dtype == torch.float32:
            configs += [(g, False, k, 0) for g, k in staged]

        def timed():
            work = workspace(self)
            Qs = Q.clone()
            rk_step(self, Qs, dt, 1, phys, work=work)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            rk_step(self, Qs, dt, steps, phys, work=work)
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / steps

        self.set_filter_launch(0, False)
        best = None
        for g, persistent, stages, pf in configs:
            self.set_persistent(persistent)
            self.set_staging(stages)
            self.set_prefetch(pf)
            self.set_launch(g, block)
            ms = timed()
            if best is None or ms < best[0]:
                best = (ms, g, persistent, stages, pf)
        _, g, persistent, stages, pf = best
        self.set_persistent(persistent)
        self.set_staging(stages)
        self.set_prefetch(pf)
        self.set_launch(g, block)
        fbest = (best[0], 0, False, block)
        for fb in filter_blocks:
            for fg in filter_groups:
                if fb % fg or fb % 32:
                    continue
                self.set_launch(g, fb)
                for fp in (False, True):
                    self.set_filter_launch(fg, fp)
                    ms = timed()
                    if ms < fbest[0]:
                        fbest = (ms, fg, fp, fb)
        block = fbest[3]
        self.set_launch(g, block)
        self.set_filter_launch(fbest[1], fbest[2])
        if self.device_status() != 0:
            raise LabfmError(7, "a staged stage kernel's bounded wait ran out while tuning")
        return {"group": g, "block": block, "persistent": persistent, "staging": stages,
                "prefetch": pf, "filter_group": fbest[1] or g, "filter_persistent": fbest[2],
                "ms_per_step": fbest[0]}

    def workspace_bytes(self) -> int:
        return int(lib.labfm_rk_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib.labfm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rhs(plan: Plan, fields: torch.Tensor, phys: Phys, out: torch.Tensor | None = None, stream=None):
    """eq. icns right-hand side of (ln rho, u, v) (labfm_rhs); fields is 3 x N."""
    fp = _state(plan, fields, "fields")
    out = torch.empty_like(fields) if out is None else out
    op = _state(plan, out, "out")
    ph = phys.c()
    _check(lib.labfm_rhs(plan.handle, fp, op, ctypes.byref(ph), _stream(stream)))
    return out


def filter(plan: Plan, fields: torch.Tensor, out: torch.Tensor | None = None, stream=None):  # noqa: A001
    """Hyperviscous filter (1 + kappa nabla^m) of the three fields (labfm_filter)."""
    fp = _state(plan, fields, "fields")
    out = torch.empty_like(fields) if out is None else out
    _check(lib.labfm_filter(plan.handle, fp, _state(plan, out, "out"), _stream(stream)))
    return out


def save_operator(path: str, row_ptr, col, w, kappa, s, **meta) -> None:
    """Write a built operator (the inputs of labfm_plan_create: CSR row_ptr and col,
    the FP64 weights (6, nnz), kappa and s) with any scalar metadata to one .npz
    file, so that a run can resume without the neighbour search and weight build."""
    import numpy as np
    arrays = {k: t.detach().cpu().numpy() for k, t in
              (("row_ptr", row_ptr), ("col", col), ("w", w), ("kappa", kappa), ("s", s))}
    np.savez(path, **arrays, meta_keys=np.array(sorted(meta), dtype=object),
             meta_values=np.array([meta[k] for k in sorted(meta)], dtype=object))


def load_operator(path: str, device="cuda") -> dict:
    """The operator save_operator wrote, as tensors on `device` (row_ptr, col, w,
    kappa, s) plus its metadata under "meta"."""
    import numpy as np
    with np.load(path, allow_pickle=True) as f:
        out = {k: torch.from_numpy(f[k]).to(device) for k in ("row_ptr", "col", "w", "kappa", "s")}
        out["meta"] = dict(zip(f["meta_keys"].tolist(), f["meta_values"].tolist()))
    return out


def save_state(path: str, Q, step: int, t: float, dt: float, **meta) -> None:
    """A checkpoint of the evolved state (ln rho, u, v) after `step` steps at time t
    with time step dt (and scalar metadata), as one .npz file."""
    import numpy as np
    np.savez(path, Q=Q.detach().cpu().numpy(), step=np.int64(step), t=np.float64(t), dt=np.float64(dt),
             meta_keys=np.array(sorted(meta), dtype=object),
             meta_values=np.array([meta[k] for k in sorted(meta)], dtype=object))


def load_state(path: str, device="cuda") -> dict:
    """The checkpoint save_state wrote: Q on `device`, step, t, dt and "meta"."""
    import numpy as np
    with np.load(path, allow_pickle=True) as f:
        return {"Q": torch.from_numpy(f["Q"]).to(device), "step": int(f["step"]), "t": float(f["t"]),
                "dt": float(f["dt"]), "meta": dict(zip(f["meta_keys"].tolist(), f["meta_values"].tolist()))}


def workspace(plan: Plan) -> torch.Tensor:
    """A device buffer of labfm_rk_workspace_bytes for rk_step."""
    nb = plan.workspace_bytes()
    return torch.empty(max(nb, 16), dtype=torch.uint8, device=plan.device)


def rk_step(plan: Plan, Q: torch.Tensor, dt: float, nsteps: int, phys: Phys,
            work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """nsteps RK3(2)4[2R+]C steps + filter, in place on Q (labfm_rk_step)."""
    qp = _state(plan, Q)
    work = workspace(plan) if work is None else work
    ph = phys.c()
    _check(lib.labfm_rk_step(plan.handle, qp, _ptr(work), work.numel(), float(dt), int(nsteps),
                             ctypes.byref(ph), _stream(stream)))
    return Q


def stable_dt(plan: Plan, fields: torch.Tensor, s: torch.Tensor, c: float, mu: float,
              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """eq. dt as a 1-element float64 device tensor (labfm_stable_dt)."""
    _nodes(plan, s, "s")
    fp, sp = _state(plan, fields, "fields"), _ptr(s)
    out = torch.empty(1, dtype=torch.float64, device=fields.device) if out is None else out
    _check(lib.labfm_stable_dt(plan.handle, fp, sp, float(c), float(mu), _ptr(out),
                               _stream(stream)))
    return out


def rk_step_host(plan: Plan, Q_host: torch.Tensor, Q_dev: torch.Tensor, dt: float, nsteps: int,
                 phys: Phys, work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """labfm_rk_step_host: state in (pinned) host memory, copied in and out by the call."""
    if Q_host.is_cuda or not Q_host.is_contiguous():
        raise ValueError("Q_host must be a contiguous host tensor")
    if Q_host.dtype != plan.dtype or tuple(Q_host.shape) != (3, plan.N):
        raise ValueError(f"Q_host must be {plan.dtype} of shape (3, {plan.N})")
    qd = _state(plan, Q_dev, "Q_dev")
    work = workspace(plan) if work is None else work
    ph = phys.c()
    _check(lib.labfm_rk_step_host(plan.handle, Q_host.data_ptr(), qd, _ptr(work), work.numel(),
                                  float(dt), int(nsteps), ctypes.byref(ph), _stream(stream)))
    return Q_host


def probe_fma_rate(dtype=torch.float64) -> float:
    """Device FMA throughput in GFLOP/s for float64 or float32 (labfm_probe_fma_rate)."""
    out = _D(0.0)
    _check(lib.labfm_probe_fma_rate(LABFM_F64 if dtype == torch.float64 else LABFM_F32,
                                    ctypes.byref(out)))
    return out.value


def rk_step_noalloc(plan: Plan, Q: torch.Tensor, dt: float, nsteps: int, phys: Phys,
                    stream=None) -> torch.Tensor:
    """labfm_rk_step_noalloc: rk_step without a work buffer, for callers that cannot
    allocate device memory; the state buffers live in the library's static device
    array (16 MiB: N <= 349,525 in float32 (349,524 for a persistent plan),
    <= 174,762 in float64)."""
    qp = _state(plan, Q)
    ph = phys.c()
    _check(lib.labfm_rk_step_noalloc(plan.handle, qp, float(dt), int(nsteps), ctypes.byref(ph),
                                     _stream(stream)))
    return Q


class StepGraph:
    """labfm_step_graph_*: one captured CUDA graph per time step, replayed per step."""

    def __init__(self, plan: Plan, dt: float, phys: Phys, work: torch.Tensor | None = None):
        self.plan = plan
        self.work = workspace(plan) if work is None else work
        self._phys = phys.c()
        h = _P()
        _check(lib.labfm_step_graph_create(ctypes.byref(h), plan.handle, _ptr(self.work),
                                           self.work.numel(), float(dt), ctypes.byref(self._phys)))
        self._h = h

    def run(self, Q: torch.Tensor, nsteps: int, stream=None) -> torch.Tensor:
        _check(lib.labfm_step_graph_run(self._h, _state(self.plan, Q), int(nsteps), _stream(stream)))
        return Q

    def close(self):
        if getattr(self, "_h", None):
            lib.labfm_step_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- adjoint

def _dcode(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return LABFM_F32
    if t.dtype == torch.float64:
        return LABFM_F64
    raise ValueError("float32 or float64 tensors only")


def enable_adjoint(plan: Plan, stream=None) -> None:
    """labfm_plan_enable_adjoint: build the transposed operator of the plan."""
    _check(lib.labfm_plan_enable_adjoint(plan.handle, _stream(stream)))


def adjoint_workspace(plan: Plan) -> torch.Tensor:
    nb = int(lib.labfm_adjoint_workspace_bytes(plan.handle))
    return torch.empty(max(nb, 16), dtype=torch.uint8, device=plan.device)


def rhs_adjoint(plan: Plan, fields, lam, phys: Phys, work=None, stream=None):
    """(dR/dq)^T lam at state `fields` (labfm_rhs_adjoint)."""
    fp, lp = _state(plan, fields, "fields"), _state(plan, lam, "lam")
    work = adjoint_workspace(plan) if work is None else work
    out = torch.empty_like(fields)
    ph = phys.c()
    _check(lib.labfm_rhs_adjoint(plan.handle, fp, lp, _ptr(out), ctypes.byref(ph),
                                 _ptr(work), work.numel(), _stream(stream)))
    return out


def rk_step_adjoint(plan: Plan, Q, lam, dt: float, phys: Phys, work=None, stream=None):
    """lam <- (dQ_next/dQ)^T lam for one step from state Q (labfm_rk_step_adjoint), in place."""
    qp, lp = _state(plan, Q), _state(plan, lam, "lam")
    work = adjoint_workspace(plan) if work is None else work
    ph = phys.c()
    _check(lib.labfm_rk_step_adjoint(plan.handle, qp, lp, float(dt), ctypes.byref(ph),
                                     _ptr(work), work.numel(), _stream(stream)))
    return lam


def stage_states(plan: Plan) -> torch.Tensor:
    """A buffer for the four packed stage states of one step (labfm_stage_states_bytes)."""
    nb = int(lib.labfm_stage_states_bytes(plan.handle))
    return torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=plan.device)


def rk_step_record(plan: Plan, Q, states, dt: float, phys: Phys, work=None, stream=None):
    """labfm_rk_step_record: Q advanced one step in place, its stage states kept in `states`."""
    qp = _state(plan, Q)
    work = workspace(plan) if work is None else work
    ph = phys.c()
    _check(lib.labfm_rk_step_record(plan.handle, qp, _ptr(states), states.numel(), _ptr(work),
                                    work.numel(), float(dt), ctypes.byref(ph), _stream(stream)))
    return Q


def rk_step_adjoint_recorded(plan: Plan, states, lam, dt: float, phys: Phys, work=None, stream=None):
    """lam <- (dQ_next/dQ)^T lam from recorded stage states (labfm_rk_step_adjoint_recorded)."""
    lp = _state(plan, lam, "lam")
    work = adjoint_workspace(plan) if work is None else work
    ph = phys.c()
    _check(lib.labfm_rk_step_adjoint_recorded(plan.handle, _ptr(states), lp, float(dt),
                                              ctypes.byref(ph), _ptr(work), work.numel(), _stream(stream)))
    return lam


def filter_adjoint(plan: Plan, lam, work=None, stream=None):
    lp = _state(plan, lam, "lam")
    work = adjoint_workspace(plan) if work is None else work
    out = torch.empty_like(lam)
    _check(lib.labfm_filter_adjoint(plan.handle, lp, _ptr(out), _ptr(work), work.numel(),
                                    _stream(stream)))
    return out


def conserved_to_primitive(c, stream=None):
    _field_dtype(c, "c")
    q = torch.empty_like(c)
    _check(lib.labfm_conserved_to_primitive(_ptr(c), _ptr(q), c.shape[1], _dcode(c), _stream(stream)))
    return q


def conserved_vjp(c, qbar, stream=None):
    _field_dtype(c, "c")
    _check_tensor(qbar, c.dtype, tuple(c.shape), "qbar")
    cb = torch.empty_like(c)
    _check(lib.labfm_conserved_vjp(_ptr(c), _ptr(qbar), _ptr(cb), c.shape[1], _dcode(c),
                                   _stream(stream)))
    return cb


def kinetic_energy(q, s, stream=None) -> torch.Tensor:
    _check_tensor(s, torch.float64, (_field_dtype(q, "q"),), "s")
    out = torch.empty(1, dtype=torch.float64, device=q.device)
    _check(lib.labfm_kinetic_energy(_ptr(q), _ptr(s), q.shape[1], _dcode(q), _ptr(out), _stream(stream)))
    return out


def kinetic_energy_grad(q, s, scale: float = 1.0, stream=None):
    _check_tensor(s, torch.float64, (_field_dtype(q, "q"),), "s")
    g = torch.empty_like(q)
    _check(lib.labfm_kinetic_energy_grad(_ptr(q), _ptr(s), q.shape[1], _dcode(q), float(scale), _ptr(g),
                                         _stream(stream)))
    return g


def probe_momentum(q, px, py, stream=None) -> torch.Tensor:
    """labfm_probe_momentum: sum_i rho_i (px_i u_i + py_i v_i), 1-element float64 tensor."""
    N = _field_dtype(q, "q")
    _check_tensor(px, torch.float64, (N,), "px")
    _check_tensor(py, torch.float64, (N,), "py")
    out = torch.empty(1, dtype=torch.float64, device=q.device)
    _check(lib.labfm_probe_momentum(_ptr(q), _ptr(px), _ptr(py), q.shape[1], _dcode(q), _ptr(out),
                                    _stream(stream)))
    return out


def probe_momentum_grad(q, px, py, scale: float = 1.0, stream=None):
    N = _field_dtype(q, "q")
    _check_tensor(px, torch.float64, (N,), "px")
    _check_tensor(py, torch.float64, (N,), "py")
    g = torch.empty_like(q)
    _check(lib.labfm_probe_momentum_grad(_ptr(q), _ptr(px), _ptr(py), q.shape[1], _dcode(q), float(scale),
                                         _ptr(g), _stream(stream)))
    return g


class _Rollout(torch.autograd.Function):
    """nsteps time steps of a plan as a differentiable map q0 -> q_final.

    Forward keeps a checkpoint of the state every `every` steps, and records the
    stage states of the last segment as it steps through it (labfm_rk_step_record,
    the same arithmetic as labfm_rk_step), so that backward need not recompute
    that segment.  Backward walks the segments last to first: it recomputes each
    earlier segment from its checkpoint with labfm_rk_step_record, keeping every
    step's stage states, then applies labfm_rk_step_adjoint_recorded step by step
    in reverse."""

    @staticmethod
    def forward(ctx, q0, plan, dt, nsteps, phys, every):
        work = workspace(plan)
        q = q0.detach().clone()
        ckpts = []
        # without a gradient to take (no_grad, or q0 not requiring one) nothing is recorded
        last = ((nsteps - 1) // every) * every if (nsteps > 0 and ctx.needs_input_grad[0]) else nsteps
        recorded = []
        for k in range(nsteps):
            if k % every == 0:
                ckpts.append(q.clone())
            if k >= last:
                X = stage_states(plan)
                rk_step_record(plan, q, X, dt, phys, work=work)
                recorded.append(X)
            else:
                rk_step(plan, q, dt, 1, phys, work=work)
        ctx.plan, ctx.dt, ctx.nsteps, ctx.phys, ctx.every = plan, dt, nsteps, phys, every
        ctx.ckpts = ckpts
        ctx.recorded_last = recorded
        return q

    @staticmethod
    def backward(ctx, gq):
        plan, dt, nsteps, phys, every = ctx.plan, ctx.dt, ctx.nsteps, ctx.phys, ctx.every
        lam = gq.detach().clone().contiguous()
        work = workspace(plan)
        awork = adjoint_workspace(plan)
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            if seg == len(ctx.ckpts) - 1:
                recorded = ctx.recorded_last  # recorded by the forward pass
                ctx.recorded_last = None
            else:
                k0 = seg * every
                k1 = min(nsteps, k0 + every)
                q = ctx.ckpts[seg].clone()
                recorded = []
                for _ in range(k0, k1):
                    X = stage_states(plan)
                    rk_step_record(plan, q, X, dt, phys, work=work)
                    recorded.append(X)
            for X in reversed(recorded):
                rk_step_adjoint_recorded(plan, X, lam, dt, phys, work=awork)
            recorded = None
        ctx.ckpts = None
        return lam, None, None, None, None, None


def rollout(plan: Plan, q0: torch.Tensor, dt: float, nsteps: int, phys: Phys,
            checkpoint_every: int = 50) -> torch.Tensor:
    """Differentiable nsteps-step rollout of the evolved state (ln rho, u, v).
    Requires enable_adjoint(plan) before backward."""
    return _Rollout.apply(q0, plan, dt, nsteps, phys, checkpoint_every)


class _ToPrimitive(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c):
        ctx.save_for_backward(c)
        return conserved_to_primitive(c.detach().contiguous())

    @staticmethod
    def backward(ctx, qbar):
        (c,) = ctx.saved_tensors
        return conserved_vjp(c.detach().contiguous(), qbar.contiguous())


class _KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, s):
        ctx.save_for_backward(q, s)
        return kinetic_energy(q.detach().contiguous(), s)

    @staticmethod
    def backward(ctx, g):
        q, s = ctx.saved_tensors
        grad = kinetic_energy_grad(q.detach().contiguous(), s, float(g.sum().item()))
        return grad, None


class _ProbeMomentum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, px, py):
        ctx.save_for_backward(q, px, py)
        return probe_momentum(q.detach().contiguous(), px, py)

    @staticmethod
    def backward(ctx, g):
        q, px, py = ctx.saved_tensors
        return probe_momentum_grad(q.detach().contiguous(), px, py, float(g.sum().item())), None, None


def to_primitive(c: torch.Tensor) -> torch.Tensor:
    """Differentiable (rho, rho u, rho v) -> (ln rho, u, v)."""
    return _ToPrimitive.apply(c)


def domain_kinetic_energy(q: torch.Tensor, s: torch.Tensor) -> torch.Tensor:
    """Differentiable sum_i 1/2 rho |u|^2 s_i^2 (1-element float64 tensor)."""
    return _KineticEnergy.apply(q, s)


def domain_probe_momentum(q: torch.Tensor, px: torch.Tensor, py: torch.Tensor) -> torch.Tensor:
    """Differentiable sum_i rho_i (px_i u_i + py_i v_i) (1-element float64 tensor)."""
    return _ProbeMomentum.apply(q, px, py)
