"""cp_gradient_all_noalloc: the all-mode gradient for callers that cannot
allocate device memory (a plugin whose host application owns every device
allocation, or code that must not call cudaMalloc after start-up).  It takes
its scratch from a fixed array inside the library; its results must match
the FP64 oracle and equal those of cp_gradient_all with a caller workspace,
call after call, and device-side conditions recorded in the array's status
word must reach the caller (cpg_noalloc_scratch + cpg_device_status).

This file is collected last, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import cpsynth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CPG_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as m
    L = m.lib()
    L.cp_gradient_all_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p]
    L.cp_gradient_all_noalloc.restype = ctypes.c_int
    L.cpg_noalloc_scratch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t)]
    L.cpg_noalloc_scratch.restype = ctypes.c_int
    return m


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _scratch_opts(cg):
    """cpg_opts naming the fixed array as the workspace (for the status calls)."""
    ptr, nbytes = ctypes.c_void_p(), ctypes.c_size_t()
    assert cg.lib().cpg_noalloc_scratch(ctypes.byref(ptr), ctypes.byref(nbytes)) == 0
    assert ptr.value and nbytes.value == (64 << 20)
    return cg.cpgrad.cpg_opts(0, 0, ptr, nbytes.value, _stream())


def _noalloc(cg, Y, I, Ad, R, precision=0):
    L = cg.lib()
    I64 = (ctypes.c_int64 * len(I))(*I)
    G = [torch.full((R, In), float("nan"), device="cuda").t() for In in I]
    st = L.cp_gradient_all_noalloc(ctypes.c_void_p(Y.data_ptr()), I64, len(I), _ptrs(Ad), R, _ptrs(G), precision, 0,
                                   _stream())
    assert st == 0, st
    torch.cuda.synchronize()
    return G


def _rel(g, w):
    return float(np.linalg.norm(g.double().cpu().numpy() - w) / np.linalg.norm(w))


# [24, 20, 30, 17]: column pitch 480 floats (16-byte multiple), TMA tiles.
# [17] * 6: pitch 4913 floats; the pitched copy of Y (96 MB) does not fit in
# the 64 MB array while the rest of the scratch does, so Y is streamed itself.
@pytest.mark.parametrize("I,R", [([24, 20, 30, 17], 12), ([17] * 6, 6)])
def test_noalloc_matches_oracle_and_workspace_call(cg, I, R):
    y = cpsynth.random_tensor(I, seed=21)
    A = cpsynth.random_factors(I, R, seed=21)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    ref = [g.clone() for g in cg.cp_gradient_all(Y, I, Ad)]
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the fixed scratch
        G = _noalloc(cg, Y, I, Ad, R)
        for n, g in enumerate(G):
            assert _rel(g, want[n]) <= 1e-5, (n, _rel(g, want[n]))
            assert _rel(g, ref[n].double().cpu().numpy()) <= 1e-5
    assert cg.lib().cpg_device_status(ctypes.byref(_scratch_opts(cg))) == 0


@pytest.mark.parametrize("prec", [2, 5])  # CPG_BF16X3, CPG_BF16X6
def test_noalloc_split_precision(cg, prec):
    I, R = [24, 20, 30, 17], 12
    y = cpsynth.random_tensor(I, seed=22)
    A = cpsynth.random_factors(I, R, seed=22)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for _ in range(2):
        G = _noalloc(cg, Y, I, Ad, R, precision=prec)
        for n, g in enumerate(G):
            assert _rel(g, want[n]) <= 1e-5, (prec, n)
    assert cg.lib().cpg_device_status(ctypes.byref(_scratch_opts(cg))) == 0


def test_noalloc_status_is_kept_until_read(cg):
    """A bounded wait that expires on the array (the self-test) is still
    reported after a later no-allocation call, then cleared by the read."""
    L = cg.lib()
    o = _scratch_opts(cg)
    assert L.cpg_device_status(ctypes.byref(o)) == 0
    assert L.cpg_selftest_timeout(ctypes.byref(o), 64) == 0
    I, R = [12, 10, 14], 4
    y = cpsynth.random_tensor(I, seed=23)
    A = cpsynth.random_factors(I, R, seed=23)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    G = _noalloc(cg, Y, I, Ad, R)
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    assert all(_rel(g, w) <= 1e-5 for g, w in zip(G, want))
    assert L.cpg_device_status(ctypes.byref(o)) == CPG_ERR_TIMEOUT
    assert L.cpg_device_status(ctypes.byref(o)) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(cg):
    L = cg.lib()
    I = [1000, 1000, 1000]          # workspace needed is far above the fixed array
    I64 = (ctypes.c_int64 * 3)(*I)
    dummy = ctypes.c_void_p(256)
    P = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    assert cg.cpg_workspace_size(I, 64) > (64 << 20)
    assert L.cp_gradient_all_noalloc(dummy, I64, 3, P, 64, P, 0, 0, None) == 3   # CPG_ERR_WORKSPACE
    # argument errors first, as cp_gradient_all returns them
    assert L.cp_gradient_all_noalloc(None, I64, 3, P, 64, P, 0, 0, None) == 1   # CPG_ERR_ARG
    big = (ctypes.c_int64 * 3)(1 << 40, 1 << 40, 1 << 40)
    assert L.cp_gradient_all_noalloc(dummy, big, 3, P, 4, P, 0, 0, None) == 2   # CPG_ERR_SHAPE
