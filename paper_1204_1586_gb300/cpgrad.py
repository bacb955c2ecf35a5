"""Python binding of libcpgrad.so: argument marshalling only.

Every step of the computation runs in the CUDA library behind the C ABI
declared in ``include/cpgrad.h``; this module only checks tensor layouts,
allocates outputs and workspace with PyTorch, and passes device pointers
and the current CUDA stream.  There is no CPU fallback: if the library is
missing, importing the low-level handle raises.

Layouts (as in the C ABI): vec(Y) is a 1-D tensor with mode 1 fastest
(eq. 2.1); factor A^(n) and gradient G^(n) are (I_n, R) tensors stored
column-major (stride (1, I_n)); ``colmajor()`` converts.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpgrad.so")

CPG_OK, CPG_ERR_ARG, CPG_ERR_SHAPE, CPG_ERR_WORKSPACE, CPG_ERR_SINGULAR, CPG_ERR_CUDA, CPG_ERR_TIMEOUT, \
    CPG_ERR_UNSUPPORTED = range(8)
PRECISIONS = {"fp32": 0, "tf32x3": 1, "bf16x3": 2, "bf16": 3, "fp64": 4, "bf16x6": 5}
CALL_GRADIENT_ALL, CALL_GRADIENT_MODE, CALL_ALS, CALL_GRADIENT_TUNE, CALL_GRADIENT_FULL, CALL_NTF, CALL_ALS_TUNE = \
    range(7)
EXPORTS = ["cpg_split_point", "cpg_workspace_size", "cp_gradient_all", "cp_gradient_mode", "cp_als_iter",
           "cpg_workspace_size_batched", "cp_als_batched", "cpg_workspace_init", "cpg_device_status", "cpg_status_str",
           "cpg_launch_count", "cpg_profile_lead", "cpg_profile_read", "cpg_autotune_gradient",
           "cpg_gradient_plan_query", "cpg_autotune_clear", "cp_gradient_full", "cp_gradient_step", "cp_ntf_iter",
           "cpg_selftest_timeout", "cpg_als_candidates", "cpg_autotune_als", "cpg_als_plan_query",
           "cpg_gradient_plan_set", "cpg_als_plan_set"]


class CpgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} (status {status})")
        self.status = status


class cpg_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("split", ctypes.c_int), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p)]


class cpg_gradient_plan(ctypes.Structure):
    _fields_ = [("split", ctypes.c_int), ("fused", ctypes.c_int), ("ms", ctypes.c_float), ("candidates", ctypes.c_int)]


class cpg_als_plan(ctypes.Structure):
    _fields_ = [("split", ctypes.c_int), ("ms", ctypes.c_float), ("candidates", ctypes.c_int)]


class cpg_tensor_desc(ctypes.Structure):
    _fields_ = [("Y", ctypes.c_void_p), ("N", ctypes.c_int), ("I", ctypes.POINTER(ctypes.c_int64)),
                ("A", ctypes.POINTER(ctypes.c_void_p)), ("lam", ctypes.c_void_p), ("R", ctypes.c_int),
                ("fit", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcpgrad.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vpp = ctypes.POINTER(ctypes.c_void_p)
        L.cpg_split_point.argtypes = [i64p, ctypes.c_int]
        L.cpg_split_point.restype = ctypes.c_int
        L.cpg_workspace_size.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts), ctypes.c_int]
        L.cpg_workspace_size.restype = ctypes.c_size_t
        L.cp_gradient_all.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, vpp,
                                      ctypes.POINTER(cpg_opts)]
        L.cp_gradient_all.restype = ctypes.c_int
        L.cp_gradient_mode.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.POINTER(cpg_opts)]
        L.cp_gradient_mode.restype = ctypes.c_int
        L.cp_als_iter.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(cpg_opts)]
        L.cp_als_iter.restype = ctypes.c_int
        L.cpg_workspace_size_batched.argtypes = [ctypes.c_int, ctypes.POINTER(cpg_tensor_desc),
                                                 ctypes.POINTER(cpg_opts)]
        L.cpg_workspace_size_batched.restype = ctypes.c_size_t
        L.cp_als_batched.argtypes = [ctypes.c_int, ctypes.POINTER(cpg_tensor_desc), ctypes.c_int,
                                     ctypes.POINTER(cpg_opts)]
        L.cp_als_batched.restype = ctypes.c_int
        L.cpg_workspace_init.argtypes = [ctypes.POINTER(cpg_opts)]
        L.cpg_workspace_init.restype = ctypes.c_int
        L.cpg_device_status.argtypes = [ctypes.POINTER(cpg_opts)]
        L.cpg_device_status.restype = ctypes.c_int
        L.cpg_status_str.argtypes = [ctypes.c_int]
        L.cpg_status_str.restype = ctypes.c_char_p
        L.cpg_launch_count.argtypes = [ctypes.c_int]
        L.cpg_launch_count.restype = ctypes.c_uint64
        L.cpg_profile_lead.argtypes = [ctypes.c_int]
        L.cpg_profile_lead.restype = ctypes.c_int
        L.cpg_profile_read.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.cpg_profile_read.restype = ctypes.c_int
        L.cpg_autotune_gradient.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, vpp,
                                            ctypes.POINTER(cpg_opts), ctypes.c_int, ctypes.POINTER(cpg_gradient_plan)]
        L.cpg_autotune_gradient.restype = ctypes.c_int
        L.cpg_gradient_plan_query.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts),
                                              ctypes.POINTER(cpg_gradient_plan)]
        L.cpg_gradient_plan_query.restype = ctypes.c_int
        L.cpg_autotune_clear.argtypes = []
        L.cpg_autotune_clear.restype = None
        L.cpg_als_candidates.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.cpg_als_candidates.restype = ctypes.c_int
        L.cpg_autotune_als.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(cpg_opts), ctypes.c_int, ctypes.POINTER(cpg_als_plan)]
        L.cpg_autotune_als.restype = ctypes.c_int
        L.cpg_als_plan_query.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts),
                                         ctypes.POINTER(cpg_als_plan)]
        L.cpg_als_plan_query.restype = ctypes.c_int
        L.cpg_gradient_plan_set.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts),
                                            ctypes.POINTER(cpg_gradient_plan)]
        L.cpg_gradient_plan_set.restype = ctypes.c_int
        L.cpg_als_plan_set.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cpg_opts),
                                       ctypes.POINTER(cpg_als_plan)]
        L.cpg_als_plan_set.restype = ctypes.c_int
        L.cp_gradient_full.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, vpp,
                                       ctypes.POINTER(cpg_opts)]
        L.cp_gradient_full.restype = ctypes.c_int
        L.cp_gradient_step.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, ctypes.c_double, vpp,
                                       ctypes.POINTER(cpg_opts)]
        L.cp_gradient_step.restype = ctypes.c_int
        L.cp_ntf_iter.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int, vpp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.POINTER(cpg_opts)]
        L.cp_ntf_iter.restype = ctypes.c_int
        L.cpg_selftest_timeout.argtypes = [ctypes.POINTER(cpg_opts), ctypes.c_uint]
        L.cpg_selftest_timeout.restype = ctypes.c_int
        _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().cpg_status_str(int(status)).decode()


def _i64(I: Sequence[int]):
    return (ctypes.c_int64 * len(I))(*[int(v) for v in I])


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


def _prec(precision) -> int:
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def cpg_split_point(I: Sequence[int]) -> int:
    return int(lib().cpg_split_point(_i64(I), len(I)))


def cpg_workspace_size(I: Sequence[int], R: int, precision="fp32", split: int = 0, call: int = CALL_GRADIENT_ALL) -> int:
    o = cpg_opts(_prec(precision), int(split), None, 0, None)
    return int(lib().cpg_workspace_size(_i64(I), len(I), int(R), ctypes.byref(o), int(call)))


def launch_count(reset: bool = False) -> int:
    return int(lib().cpg_launch_count(1 if reset else 0))


# Launch kinds of the timing record (cpgrad.h CPG_KIND_*).
LAUNCH_KINDS = {1: "lead_step4_R", 2: "lead_step7_L", 3: "lead_step4+7_fused", 10: "chain_segmented_dot",
                11: "als_mode_fused_update", 12: "gram", 13: "kronecker_vector", 14: "norm_y2",
                15: "als_update_fp64_or_ntf", 16: "gradient_model_term", 17: "khatri_rao_rows",
                18: "pitched_copy_of_y"}


def profile_lead(enable) -> None:
    """Event timing of launches: True / 1 = leading passes only, 2 = every
    kernel of the library, False / 0 = stop."""
    mode = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
    st = lib().cpg_profile_lead(mode)
    if st != CPG_OK:
        raise CpgError(st, "cpg_profile_lead")


def profile_read(max_entries: int = 4096):
    """[(milliseconds, kind)] of the launches recorded since profile_lead(...), in launch order."""
    ms = (ctypes.c_float * max_entries)()
    sd = (ctypes.c_int * max_entries)()
    n = lib().cpg_profile_read(ms, sd, max_entries)
    if n < 0:
        raise CpgError(CPG_ERR_CUDA, "cpg_profile_read")
    return [(float(ms[i]), int(sd[i])) for i in range(n)]


# ---- torch-facing helpers -------------------------------------------------------------
def _torch():
    import torch
    return torch


def colmajor(A):
    """(I, R) tensor with column-major storage (stride (1, I))."""
    return A.t().contiguous().t()


def _check_colmajor(A, In, R, dtype, name):
    if tuple(A.shape) != (In, R) or A.dtype != dtype or not A.is_cuda:
        raise ValueError(f"{name}: expected a CUDA {dtype} tensor of shape ({In}, {R}), got {tuple(A.shape)} {A.dtype}")
    if A.numel() > 0 and not (A.stride(0) == 1 and (R == 1 or A.stride(1) == In)):
        raise ValueError(f"{name}: must be column-major (stride (1, {In})); use colmajor()")


class Workspace:
    """Device scratch for the library, held as a torch uint8 tensor and grown on demand."""

    def __init__(self, device=None):
        self.buf = None
        self.device = device

    def get(self, nbytes: int, stream_ptr):
        torch = _torch()
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device or "cuda")
            o = cpg_opts(0, 0, ctypes.c_void_p(self.buf.data_ptr()), self.buf.numel(), ctypes.c_void_p(stream_ptr))
            st = lib().cpg_workspace_init(ctypes.byref(o))
            if st != CPG_OK:
                raise CpgError(st, "cpg_workspace_init")
        return self.buf


_default_ws = {}


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _opts(precision, split, ws: Workspace, nbytes, stream_ptr):
    buf = ws.get(nbytes, stream_ptr)
    return cpg_opts(_prec(precision), int(split), ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                    ctypes.c_void_p(stream_ptr))


def _dev_key(device):
    torch = _torch()
    d = torch.device(device) if device is not None else torch.device("cuda")
    if d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return d


def _ws_for(workspace, device):
    if workspace is not None:
        return workspace
    d = _dev_key(device)
    key = str(d)
    if key not in _default_ws:
        _default_ws[key] = Workspace(d)
    return _default_ws[key]


def _check_y(Y, I, dtype):
    n = 1
    for v in I:
        n *= int(v)
    if not Y.is_cuda or Y.dtype != dtype or Y.numel() != n or not Y.is_contiguous():
        raise ValueError(f"Y: expected a contiguous CUDA {dtype} tensor with {n} elements (vec(Y), mode 1 fastest)")


def cp_gradient_all(Y, I: Sequence[int], A, G=None, *, precision="fp32", split: int = 0, workspace=None,
                    stream=None):
    """All-mode CP gradient (Algorithm 2).  Returns the list of G^(n) (I_n x R, column-major)."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for n, a in enumerate(A):
        _check_colmajor(a, int(I[n]), R, dtype, f"A[{n}]")
    if G is None:
        G = [torch.empty((R, int(In)), dtype=dtype, device=Y.device).t() for In in I]
    for n, g in enumerate(G):
        _check_colmajor(g, int(I[n]), R, dtype, f"G[{n}]")
    sp = _stream_ptr(stream)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_GRADIENT_ALL), sp)
    st = lib().cp_gradient_all(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, _ptrs(G), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_gradient_all")
    return G


def cp_gradient_autotune(Y, I: Sequence[int], A, G=None, *, precision="fp32", split: int = 0, reps: int = 3,
                         workspace=None, stream=None):
    """Times every plan of the all-mode gradient (split k, fused or two passes)
    on these inputs and records the fastest for later cp_gradient_all calls of
    this shape, rank and precision.  Returns {"split", "fused", "ms",
    "candidates"}; G receives the gradient."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for n, a in enumerate(A):
        _check_colmajor(a, int(I[n]), R, dtype, f"A[{n}]")
    if G is None:
        G = [torch.empty((R, int(In)), dtype=dtype, device=Y.device).t() for In in I]
    for n, g in enumerate(G):
        _check_colmajor(g, int(I[n]), R, dtype, f"G[{n}]")
    sp = _stream_ptr(stream)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_GRADIENT_TUNE), sp)
    plan = cpg_gradient_plan()
    st = lib().cpg_autotune_gradient(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, _ptrs(G),
                                     ctypes.byref(o), int(reps), ctypes.byref(plan))
    if st != CPG_OK:
        raise CpgError(st, "cpg_autotune_gradient")
    return {"split": plan.split, "fused": bool(plan.fused), "ms": float(plan.ms), "candidates": plan.candidates}


def _grad_args(Y, I, A, G, precision):
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for n, a in enumerate(A):
        _check_colmajor(a, int(I[n]), R, dtype, f"A[{n}]")
    if G is None:
        G = [torch.empty((R, int(In)), dtype=dtype, device=Y.device).t() for In in I]
    for n, g in enumerate(G):
        _check_colmajor(g, int(I[n]), R, dtype, f"G[{n}]")
    return R, G


def cp_gradient_full(Y, I: Sequence[int], A, G=None, *, precision="fp32", split: int = 0, workspace=None,
                     stream=None):
    """Cost gradient of eq. 2.13 with its model term, Y_(n) KR - A^(n) Gamma^(n), every mode."""
    R, G = _grad_args(Y, I, A, G, precision)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_GRADIENT_FULL), _stream_ptr(stream))
    st = lib().cp_gradient_full(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, _ptrs(G), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_gradient_full")
    return G


def cp_gradient_step(Y, I: Sequence[int], A, eta: float, G=None, *, precision="fp32", split: int = 0,
                     workspace=None, stream=None):
    """One all-at-once first-order step (eq. 2.15): G = cost gradients at A, then A += eta G (in place)."""
    R, G = _grad_args(Y, I, A, G, precision)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_GRADIENT_FULL), _stream_ptr(stream))
    st = lib().cp_gradient_step(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, float(eta), _ptrs(G),
                                ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_gradient_step")
    return G


def cp_ntf_iter(Y, I: Sequence[int], A, iters: int, fit=None, *, precision="fp32", split: int = 0, workspace=None,
                stream=None):
    """`iters` multiplicative nonnegative CP sweeps (eq. 2.18), A updated in place; returns the fits."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for n, a in enumerate(A):
        _check_colmajor(a, int(I[n]), R, dtype, f"A[{n}]")
    if fit is None:
        fit = torch.zeros(max(int(iters), 1), dtype=torch.float64, device=Y.device)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_NTF), _stream_ptr(stream))
    st = lib().cp_ntf_iter(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, int(iters),
                           ctypes.c_void_p(fit.data_ptr()), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_ntf_iter")
    return fit


def gradient_plan(I: Sequence[int], R: int, precision="fp32", split: int = 0):
    """The recorded measured plan for this shape / rank / precision, or None."""
    o = cpg_opts(_prec(precision), int(split), None, 0, None)
    plan = cpg_gradient_plan()
    if not lib().cpg_gradient_plan_query(_i64(I), len(I), int(R), ctypes.byref(o), ctypes.byref(plan)):
        return None
    return {"split": plan.split, "fused": bool(plan.fused)}


def set_gradient_plan(I: Sequence[int], R: int, split: int, fused: bool, precision="fp32") -> None:
    """Records (split, fused) as the plan later cp_gradient_all calls of this shape / rank / precision run."""
    o = cpg_opts(_prec(precision), 0, None, 0, None)
    plan = cpg_gradient_plan(int(split), 1 if fused else 0, 0.0, 0)
    st = lib().cpg_gradient_plan_set(_i64(I), len(I), int(R), ctypes.byref(o), ctypes.byref(plan))
    if st != CPG_OK:
        raise CpgError(st, "cpg_gradient_plan_set")


def set_als_plan(I: Sequence[int], R: int, split: int, precision="fp32") -> None:
    """Records split as the CP_ALS split later sweeps of this shape / rank / precision run."""
    o = cpg_opts(_prec(precision), 0, None, 0, None)
    plan = cpg_als_plan(int(split), 0.0, 0)
    st = lib().cpg_als_plan_set(_i64(I), len(I), int(R), ctypes.byref(o), ctypes.byref(plan))
    if st != CPG_OK:
        raise CpgError(st, "cpg_als_plan_set")


def autotune_clear() -> None:
    lib().cpg_autotune_clear()


def cp_gradient_mode(Y, I: Sequence[int], A, n: int, Gn=None, *, precision="fp32", workspace=None, stream=None):
    """Single-mode CP gradient (Section 3.2)."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for m, a in enumerate(A):
        _check_colmajor(a, int(I[m]), R, dtype, f"A[{m}]")
    if Gn is None:
        Gn = torch.empty((R, int(I[n])), dtype=dtype, device=Y.device).t()
    _check_colmajor(Gn, int(I[n]), R, dtype, "Gn")
    sp = _stream_ptr(stream)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, 0, ws, cpg_workspace_size(I, R, precision, 0, CALL_GRADIENT_MODE), sp)
    st = lib().cp_gradient_mode(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), R, int(n),
                                ctypes.c_void_p(Gn.data_ptr()), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_gradient_mode")
    return Gn


def cp_als_iter(Y, I: Sequence[int], A, iters: int, lam=None, fit=None, *, precision="fp32", split: int = 0,
                workspace=None, stream=None):
    """``iters`` fast CP_ALS sweeps (Section 4); A (list of column-major factors) is updated in place.
    Returns (lambda, fit) as CUDA float64 tensors."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for m, a in enumerate(A):
        _check_colmajor(a, int(I[m]), R, dtype, f"A[{m}]")
    if lam is None:
        lam = torch.ones(R, dtype=torch.float64, device=Y.device)
    if fit is None:
        fit = torch.zeros(max(int(iters), 1), dtype=torch.float64, device=Y.device)
    sp = _stream_ptr(stream)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_ALS), sp)
    st = lib().cp_als_iter(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A), ctypes.c_void_p(lam.data_ptr()),
                           R, int(iters), ctypes.c_void_p(fit.data_ptr()), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_als_iter")
    return lam, fit


def als_candidates(I: Sequence[int], R: int, precision="fp32", split: int = 0):
    """The splits the CP_ALS autotuner times, cheapest modelled first (host only)."""
    o = cpg_opts(_prec(precision), int(split), None, 0, None)
    buf = (ctypes.c_int * 64)()
    n = lib().cpg_als_candidates(_i64(I), len(I), int(R), ctypes.byref(o), buf, 64)
    if n == 0:
        raise CpgError(CPG_ERR_ARG, "cpg_als_candidates")
    return [int(buf[i]) for i in range(min(n, 64))]


def cp_als_autotune(Y, I: Sequence[int], A, lam=None, *, precision="fp32", split: int = 0, reps: int = 2,
                    workspace=None, stream=None):
    """Times CP_ALS sweeps at each candidate split on these inputs and records
    the fastest for later cp_als_iter / cp_ntf_iter / cp_als_batched calls of
    this shape, rank and precision.  A and lam keep their entry values.
    Returns {"split", "ms", "candidates"}."""
    torch = _torch()
    R = int(A[0].shape[1])
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    _check_y(Y, I, dtype)
    for m, a in enumerate(A):
        _check_colmajor(a, int(I[m]), R, dtype, f"A[{m}]")
    if lam is None:
        lam = torch.ones(R, dtype=torch.float64, device=Y.device)
    ws = _ws_for(workspace, Y.device)
    o = _opts(precision, split, ws, cpg_workspace_size(I, R, precision, split, CALL_ALS_TUNE), _stream_ptr(stream))
    plan = cpg_als_plan()
    st = lib().cpg_autotune_als(ctypes.c_void_p(Y.data_ptr()), _i64(I), len(I), _ptrs(A),
                                ctypes.c_void_p(lam.data_ptr()), R, ctypes.byref(o), int(reps), ctypes.byref(plan))
    if st != CPG_OK:
        raise CpgError(st, "cpg_autotune_als")
    return {"split": plan.split, "ms": float(plan.ms), "candidates": plan.candidates}


def als_plan(I: Sequence[int], R: int, precision="fp32", split: int = 0):
    """The recorded measured CP_ALS split for this shape / rank / precision, or None."""
    o = cpg_opts(_prec(precision), int(split), None, 0, None)
    plan = cpg_als_plan()
    if not lib().cpg_als_plan_query(_i64(I), len(I), int(R), ctypes.byref(o), ctypes.byref(plan)):
        return None
    return plan.split


def cp_als_batched(members, iters: int, *, precision="fp32", split: int = 0, workspace=None, stream=None):
    """``iters`` fast CP_ALS sweeps on each member, all in one call.  ``members``
    is a list of (Y, I, A) or (Y, I, A, lam, fit); each A (list of column-major
    factors) is updated in place.  Returns [(lambda, fit)] per member."""
    torch = _torch()
    if len(members) == 0:
        return []
    dtype = torch.float64 if _prec(precision) == PRECISIONS["fp64"] else torch.float32
    descs = (cpg_tensor_desc * len(members))()
    keep, out = [], []
    for b, m in enumerate(members):
        Y, I, A = m[0], list(m[1]), list(m[2])
        R = int(A[0].shape[1])
        _check_y(Y, I, dtype)
        for n, a in enumerate(A):
            _check_colmajor(a, int(I[n]), R, dtype, f"member {b}: A[{n}]")
        lam = m[3] if len(m) > 3 and m[3] is not None else torch.ones(R, dtype=torch.float64, device=Y.device)
        fit = m[4] if len(m) > 4 and m[4] is not None else torch.zeros(max(int(iters), 1), dtype=torch.float64,
                                                                        device=Y.device)
        Ii, Ap = _i64(I), _ptrs(A)
        keep += [Ii, Ap]
        descs[b] = cpg_tensor_desc(ctypes.c_void_p(Y.data_ptr()), len(I), Ii, Ap, ctypes.c_void_p(lam.data_ptr()), R,
                                   ctypes.c_void_p(fit.data_ptr()))
        out.append((lam, fit))
    sp = _stream_ptr(stream)
    ws = _ws_for(workspace, members[0][0].device)
    o0 = cpg_opts(_prec(precision), int(split), None, 0, None)
    need = int(lib().cpg_workspace_size_batched(len(members), descs, ctypes.byref(o0)))
    if need == 0:
        raise CpgError(CPG_ERR_ARG, "cpg_workspace_size_batched")
    o = _opts(precision, split, ws, need, sp)
    st = lib().cp_als_batched(len(members), descs, int(iters), ctypes.byref(o))
    if st != CPG_OK:
        raise CpgError(st, "cp_als_batched")
    return out


def selftest_timeout(polls: int = 4096, workspace=None, device=None, stream=None) -> None:
    """Launch the bounded-wait self-test: a wait that can never complete gives up
    after `polls` polls and records CPG_ERR_TIMEOUT in the workspace's status word
    (read it with cpg_device_status)."""
    ws = _ws_for(workspace, device)
    o = _opts(0, 0, ws, 256, _stream_ptr(stream))
    st = lib().cpg_selftest_timeout(ctypes.byref(o), int(polls))
    if st != CPG_OK:
        raise CpgError(st, "cpg_selftest_timeout")


def cpg_device_status(workspace=None, device=None, stream=None) -> int:
    """Synchronize and read (and clear) the device status word of a workspace."""
    ws = _ws_for(workspace, device)
    if ws.buf is None:
        return CPG_OK
    o = cpg_opts(0, 0, ctypes.c_void_p(ws.buf.data_ptr()), ws.buf.numel(), ctypes.c_void_p(_stream_ptr(stream)))
    return int(lib().cpg_device_status(ctypes.byref(o)))
