"""cp_gradient_all_noalloc: the all-mode gradient for callers that cannot
allocate device memory (a plugin whose host application owns every device
allocation, or code that must not call cudaMalloc after start-up).  It takes
its scratch from a fixed array inside the library; its results must equal
those of cp_gradient_all with a caller workspace, call after call.

This file is collected last, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import cpsynth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return m


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


def test_noalloc_matches_workspace_call(cg):
    I, R = [24, 20, 30, 17], 12
    y = cpsynth.random_tensor(I, seed=21)
    A = cpsynth.random_factors(I, R, seed=21)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    want = [g.clone() for g in cg.cp_gradient_all(Y, I, Ad)]
    torch.cuda.synchronize()
    L = cg.lib()
    I64 = (ctypes.c_int64 * len(I))(*I)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the fixed scratch
        G = [torch.full((R, In), float("nan"), device="cuda").t() for In in I]
        st = L.cp_gradient_all_noalloc(ctypes.c_void_p(Y.data_ptr()), I64, len(I), _ptrs(Ad), R, _ptrs(G), 0, 0, stream)
        assert st == 0
        torch.cuda.synchronize()
        for g, w in zip(G, want):
            err = float(torch.linalg.norm((g - w).double()) / torch.linalg.norm(w.double()))
            assert err <= 1e-5, err


def test_noalloc_rejects_sizes_beyond_its_scratch(cg):
    L = cg.lib()
    I = [1000, 1000, 1000]          # workspace needed is far above the fixed array
    I64 = (ctypes.c_int64 * 3)(*I)
    dummy = ctypes.c_void_p(256)
    P = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    assert cg.cpg_workspace_size(I, 64) > (64 << 20)
    assert L.cp_gradient_all_noalloc(dummy, I64, 3, P, 64, P, 0, 0, None) == 3   # CPG_ERR_WORKSPACE
