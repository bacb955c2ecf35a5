"""CPU checks of the C ABI: the library loads without a GPU, exports every
symbol include/cpgrad.h declares, and its host-only logic (split point of
Algorithm 2 step 1, workspace sizing, argument errors) behaves as documented.
No compute entry point reaches the GPU here: every call below returns during
argument checking."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1204_1586_gb300 import cpgrad

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(cpgrad.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return cpgrad.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "cpgrad.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) - {"defined"})


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert {"cp_gradient_all", "cp_gradient_mode", "cp_als_iter"} <= set(names)
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/cpgrad.h but not exported"
    assert set(cpgrad.EXPORTS) <= set(names)


@pytest.mark.parametrize("I", [[100] * 4, [60] * 5, [15] * 7, [30, 40, 50], [100, 2], [2, 100], [2, 2], [1, 1, 1],
                               [3, 4, 5, 6, 7], [7, 6, 5, 4, 3], [1, 9, 1, 9], [64, 8, 8, 8, 8]])
def test_split_point_matches_oracle(L, I):
    assert cpgrad.cpg_split_point(I) == oracle.split_point(I)


def test_split_point_invalid(L):
    assert cpgrad.cpg_split_point([5]) == 0
    assert cpgrad.cpg_split_point([3, 0, 2]) == 0


def test_workspace_size(L):
    for call in (cpgrad.CALL_GRADIENT_ALL, cpgrad.CALL_GRADIENT_MODE, cpgrad.CALL_ALS):
        assert cpgrad.cpg_workspace_size([30, 40, 50], 5, "fp64", 0, call) > 0
        assert cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, call) > 0
        assert cpgrad.cpg_workspace_size([100] * 4, 0, "fp32", 0, call) == 0
        assert cpgrad.cpg_workspace_size([100] * 4, 10, 9, 0, call) == 0
        assert cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 4, call) == 0
    assert cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, 7) == 0
    # scratch stays well under the tensor's own size (4e8 bytes)
    a = cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_GRADIENT_ALL)
    b = cpgrad.cpg_workspace_size([100] * 4, 20, "fp32", 0, cpgrad.CALL_GRADIENT_ALL)
    assert 0 < a < 4e8 and 0 < b < 4e8


def test_workspace_counts_pitched_copy(L):
    """A tensor whose column pitch J is not a multiple of 16 bytes gets room for
    a copy of Y with a padded pitch (ALS and the two-pass gradient); one whose
    pitch already is does not."""
    for prec, esize in (("fp32", 4), ("fp64", 8)):
        q = 16 // esize
        for I, k in (([15] * 5, 2), ([9, 11, 13, 7], 1), ([13, 7, 9, 11], 1)):
            J = int(np.prod(I[:k]))
            K = int(np.prod(I[k:]))
            assert (J * esize) % 16 != 0
            copy = (J + q - 1) // q * q * K * esize
            for call in (cpgrad.CALL_ALS, cpgrad.CALL_GRADIENT_ALL):
                odd = cpgrad.cpg_workspace_size(I, 8, prec, k, call)
                assert odd >= copy, (I, prec, call)
        # the same sizes with an aligned pitch need no copy: scratch far below the tensor
        for call in (cpgrad.CALL_ALS, cpgrad.CALL_GRADIENT_ALL):
            even = cpgrad.cpg_workspace_size([16] * 5, 8, prec, 2, call)
            assert 0 < even < 16 ** 5 * esize, (prec, call)
    # a single fused pass (FP32 at rank <= 4 fuses here) reads Y once: no copy
    fused = cpgrad.cpg_workspace_size([15] * 5, 2, "fp32", 2, cpgrad.CALL_GRADIENT_ALL)
    assert fused < 15 ** 5 * 4


def _opts(prec=0, split=0, ws=None, nbytes=0):
    return cpgrad.cpg_opts(prec, split, ws, nbytes, None)


def test_argument_errors_return_before_any_launch(L):
    I = cpgrad._i64([4, 5, 6])
    dummy = ctypes.c_void_p(16)
    A = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    G = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    o = _opts()
    n0 = cpgrad.launch_count(reset=True)
    assert L.cp_gradient_all(dummy, I, 1, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG       # N < 2
    assert L.cp_gradient_all(dummy, I, 3, A, 0, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG       # R < 1
    assert L.cp_gradient_all(dummy, I, 3, A, 300, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG     # R > max
    assert L.cp_gradient_all(None, I, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG        # null Y
    assert L.cp_gradient_all(dummy, I, 3, A, 3, G, None) == cpgrad.CPG_ERR_ARG                  # null opts
    bad = (ctypes.c_void_p * 3)(dummy, None, dummy)
    assert L.cp_gradient_all(dummy, I, 3, bad, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG     # null factor
    o9 = _opts(prec=9)
    assert L.cp_gradient_all(dummy, I, 3, A, 3, G, ctypes.byref(o9)) == cpgrad.CPG_ERR_ARG      # bad precision
    o5 = _opts(split=3)
    assert L.cp_gradient_all(dummy, I, 3, A, 3, G, ctypes.byref(o5)) == cpgrad.CPG_ERR_ARG      # split = N
    Ib = cpgrad._i64([4, -1, 6])
    assert L.cp_gradient_all(dummy, Ib, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG      # I_n < 1
    Ih = cpgrad._i64([1 << 40, 1 << 40, 1 << 40])
    assert L.cp_gradient_all(dummy, Ih, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_SHAPE    # overflow
    assert L.cp_gradient_all(dummy, I, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE  # no workspace
    small = _opts(ws=dummy, nbytes=64)
    assert L.cp_gradient_all(dummy, I, 3, A, 3, G, ctypes.byref(small)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_gradient_mode(dummy, I, 3, A, 3, 3, dummy, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG  # n = N
    assert L.cp_gradient_mode(dummy, I, 3, A, 3, -1, dummy, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_gradient_mode(dummy, I, 3, A, 3, 1, None, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    lam = ctypes.c_void_p(32)
    assert L.cp_als_iter(dummy, I, 3, A, lam, 3, -1, None, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_als_iter(dummy, I, 3, A, None, 3, 2, None, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_als_iter(dummy, I, 3, A, lam, 3, 0, None, ctypes.byref(o)) == cpgrad.CPG_OK     # nothing to do
    assert L.cp_als_iter(dummy, I, 3, A, lam, 3, 2, None, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_als_iter(dummy, I, 3, A, lam, 65, 2, None, ctypes.byref(o)) == cpgrad.CPG_ERR_UNSUPPORTED
    for prec in (1, 2, 3):   # split TF32 / BF16 forms: argument checks pass, the missing workspace is reported
        op = _opts(prec=prec)
        assert L.cp_gradient_all(dummy, I, 3, A, 3, G, ctypes.byref(op)) == cpgrad.CPG_ERR_WORKSPACE
    assert cpgrad.launch_count() == n0 * 0  # nothing was launched
    assert L.cpg_workspace_init(None) == cpgrad.CPG_ERR_ARG
    assert L.cpg_device_status(None) == cpgrad.CPG_ERR_ARG


def _desc(I, R, Y=16, A=None, lam=32):
    Ii = cpgrad._i64(I)
    Ap = A if A is not None else (ctypes.c_void_p * len(I))(*([ctypes.c_void_p(16)] * len(I)))
    d = cpgrad.cpg_tensor_desc(ctypes.c_void_p(Y) if Y else None, len(I), Ii, Ap,
                               ctypes.c_void_p(lam) if lam else None, R, None)
    return d, (Ii, Ap)


def test_batched_workspace_and_argument_errors(L):
    keep = []
    members = [([4, 5, 6], 3), ([7, 3, 2, 5], 8), ([30, 40], 2)]
    descs = (cpgrad.cpg_tensor_desc * len(members))()
    for b, (I, R) in enumerate(members):
        descs[b], k = _desc(I, R)
        keep.append(k)
    o = _opts()
    total = L.cpg_workspace_size_batched(len(members), descs, ctypes.byref(o))
    each = [cpgrad.cpg_workspace_size(I, R, "fp32", 0, cpgrad.CALL_ALS) for I, R in members]
    # the shared status word plus every member's ALS workspace (256-byte aligned)
    assert total >= 256 + sum(each) and total <= 256 + sum(each) + 256 * len(members)
    assert L.cpg_workspace_size_batched(0, descs, ctypes.byref(o)) == 0
    n0 = cpgrad.launch_count(reset=True)
    assert L.cp_als_batched(len(members), descs, 2, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_als_batched(0, descs, 2, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_als_batched(len(members), descs, -1, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_als_batched(len(members), descs, 2, None) == cpgrad.CPG_ERR_ARG
    bad = (cpgrad.cpg_tensor_desc * 2)()
    bad[0], k0 = _desc([4, 5, 6], 3)
    bad[1], k1 = _desc([4, 5, 6], 3, lam=0)     # null lambda in the second member
    assert L.cp_als_batched(2, bad, 2, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    bad[1], k1 = _desc([4, 5, 6], 65)           # rank above the ALS limit
    assert L.cp_als_batched(2, bad, 2, ctypes.byref(o)) == cpgrad.CPG_ERR_UNSUPPORTED
    bad[1], k1 = _desc([4], 3)                  # order 1
    assert L.cp_als_batched(2, bad, 2, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert cpgrad.launch_count() == 0 * n0


def test_status_strings(L):
    for s in range(8):
        assert cpgrad.status_str(s)
    assert cpgrad.status_str(99) == "unknown status"


def test_autotune_arguments_and_sizes(L):
    """The gradient autotuner checks its arguments before it launches
    anything; its workspace covers every candidate plan."""
    I = cpgrad._i64([4, 5, 6])
    dummy = ctypes.c_void_p(16)
    A = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    G = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    o = _opts()
    plan = cpgrad.cpg_gradient_plan()
    n0 = cpgrad.launch_count(reset=True)
    assert L.cpg_autotune_gradient(None, I, 3, A, 3, G, ctypes.byref(o), 3, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_gradient(dummy, I, 3, A, 3, G, ctypes.byref(o), 0, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_gradient(dummy, I, 3, A, 3, G, None, 3, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_gradient(dummy, I, 3, A, 3, G, ctypes.byref(o), 3, None) == cpgrad.CPG_ERR_WORKSPACE
    assert cpgrad.launch_count() == 0 * n0
    for I_, R in (([100] * 4, 10), ([15] * 7, 20), ([30, 40, 50], 5)):
        for prec in ("fp32", "bf16x3", "tf32x3"):
            tune = cpgrad.cpg_workspace_size(I_, R, prec, 0, cpgrad.CALL_GRADIENT_TUNE)
            assert tune >= cpgrad.cpg_workspace_size(I_, R, prec, 0, cpgrad.CALL_GRADIENT_ALL) > 0
    cpgrad.autotune_clear()
    assert cpgrad.gradient_plan([100] * 4, 10) is None


def test_als_autotune_candidates_and_sizes(L):
    """The CP_ALS autotuner's candidate splits, workspace and argument checks.
    The cost model ranks splits by the partial results of Algorithm 2's
    recursions; on the paper's cubical shapes n* (Algorithm 2 step 1) is
    always a candidate and a split that puts all but one mode on one side
    is not, once its partial result is as large as Y."""
    for I_, R in (([100] * 4, 10), ([60] * 5, 32), ([60] * 5, 64), ([15] * 7, 10), ([30, 40, 50], 5)):
        c = cpgrad.als_candidates(I_, R)
        assert oracle.split_point(I_) in c
        assert len(set(c)) == len(c) and all(1 <= k <= len(I_) - 1 for k in c)
    # 60^5: splits 1 and 4 carry a partial result of 60^4 x R, about R/60 of Y
    # twice over, far above the 1.25x margin; 2 and 3 cost the same
    assert cpgrad.als_candidates([60] * 5, 32) == [2, 3]
    # a requested split is the only candidate; a split out of range is an error
    assert cpgrad.als_candidates([60] * 5, 32, split=4) == [4]
    with pytest.raises(cpgrad.CpgError):
        cpgrad.als_candidates([60] * 5, 32, split=5)
    for I_, R in (([100] * 4, 10), ([60] * 5, 32), ([24, 20, 30, 17], 12)):
        for prec in ("fp32", "bf16x6", "tf32x3"):
            tune = cpgrad.cpg_workspace_size(I_, R, prec, 0, cpgrad.CALL_ALS_TUNE)
            als = cpgrad.cpg_workspace_size(I_, R, prec, 0, cpgrad.CALL_ALS)
            save = sum(I_) * R * 4 + R * 8
            assert tune >= als + save, (I_, R, prec)
    I = cpgrad._i64([4, 5, 6])
    dummy = ctypes.c_void_p(16)
    A = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    o = _opts()
    plan = cpgrad.cpg_als_plan()
    n0 = cpgrad.launch_count(reset=True)
    assert L.cpg_autotune_als(None, I, 3, A, dummy, 3, ctypes.byref(o), 2, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_als(dummy, I, 3, A, None, 3, ctypes.byref(o), 2, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_als(dummy, I, 3, A, dummy, 3, ctypes.byref(o), 0, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    assert L.cpg_autotune_als(dummy, I, 3, A, dummy, 3, None, 2, ctypes.byref(plan)) == cpgrad.CPG_ERR_ARG
    ob = _opts(prec=cpgrad.PRECISIONS["bf16x3"])
    assert L.cpg_autotune_als(dummy, I, 3, A, dummy, 3, ctypes.byref(ob), 2, None) == cpgrad.CPG_ERR_UNSUPPORTED
    assert L.cpg_autotune_als(dummy, I, 3, A, dummy, 3, ctypes.byref(o), 2, None) == cpgrad.CPG_ERR_WORKSPACE
    assert cpgrad.launch_count() == 0 * n0
    cpgrad.autotune_clear()
    assert cpgrad.als_plan([100] * 4, 10) is None


def test_consumer_entry_points_check_arguments(L):
    """cp_gradient_full / cp_gradient_step / cp_ntf_iter return argument and
    workspace errors before launching anything."""
    I = cpgrad._i64([4, 5, 6])
    dummy = ctypes.c_void_p(16)
    A = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    G = (ctypes.c_void_p * 3)(dummy, dummy, dummy)
    o = _opts()
    n0 = cpgrad.launch_count(reset=True)
    assert L.cp_gradient_full(None, I, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_gradient_full(dummy, I, 3, A, 3, None, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_gradient_full(dummy, I, 3, A, 3, G, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_gradient_step(dummy, I, 3, A, 3, float("nan"), G, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_gradient_step(dummy, I, 3, A, 3, 0.1, G, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_ntf_iter(dummy, I, 3, A, 3, -1, None, ctypes.byref(o)) == cpgrad.CPG_ERR_ARG
    assert L.cp_ntf_iter(dummy, I, 3, A, 3, 0, None, ctypes.byref(o)) == cpgrad.CPG_OK    # nothing to do
    assert L.cp_ntf_iter(dummy, I, 3, A, 3, 2, None, ctypes.byref(o)) == cpgrad.CPG_ERR_WORKSPACE
    assert L.cp_ntf_iter(dummy, I, 3, A, 65, 2, None, ctypes.byref(o)) == cpgrad.CPG_ERR_UNSUPPORTED
    assert cpgrad.launch_count() == 0 * n0
    full = cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_GRADIENT_FULL)
    assert full > cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_GRADIENT_ALL)
    assert cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_NTF) == \
        cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_ALS)


def test_selftest_timeout_arguments(L):
    dummy = ctypes.c_void_p(256)
    n0 = cpgrad.launch_count(reset=True)
    assert L.cpg_selftest_timeout(None, 16) == cpgrad.CPG_ERR_ARG
    assert L.cpg_selftest_timeout(ctypes.byref(_opts()), 16) == cpgrad.CPG_ERR_ARG            # no workspace
    assert L.cpg_selftest_timeout(ctypes.byref(_opts(ws=dummy, nbytes=64)), 16) == cpgrad.CPG_ERR_ARG
    assert L.cpg_selftest_timeout(ctypes.byref(_opts(ws=dummy, nbytes=256)), 0) == cpgrad.CPG_ERR_ARG
    assert L.cpg_selftest_timeout(ctypes.byref(_opts(ws=dummy, nbytes=256)), (1 << 24) + 1) == cpgrad.CPG_ERR_ARG
    assert cpgrad.launch_count() == 0 * n0


def test_noalloc_bound_leaves_out_the_pitched_copy(L):
    """The no-allocation entry point's fixed 64 MB scratch need not hold the
    optional pitched copy of Y: a 17^6 tensor (column pitch 4913 floats at
    the split k = 3) asks 96 MB more than that for the copy, yet its other
    scratch fits, so the call passes the size check.  Without a GPU it then
    fails at the device query with CPG_ERR_CUDA, launching nothing."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("dummy pointers: this check runs only where no GPU can be reached")
    I = [17] * 6
    assert cpgrad.cpg_workspace_size(I, 6) > (64 << 20)
    I64 = (ctypes.c_int64 * 6)(*I)
    dummy = ctypes.c_void_p(256)
    P = (ctypes.c_void_p * 6)(*([dummy] * 6))
    st = L.cp_gradient_all_noalloc(dummy, I64, 6, P, 6, P, 0, 0, None)
    assert st != cpgrad.CPG_ERR_WORKSPACE
    assert st == cpgrad.CPG_ERR_CUDA


def test_plan_set_arguments(L):
    """Recorded plans: a valid one is read back, an invalid split or an
    unsupported fused plan is refused, and clearing forgets both kinds."""
    cpgrad.autotune_clear()
    cpgrad.set_gradient_plan([100] * 4, 10, 3, True)
    assert cpgrad.gradient_plan([100] * 4, 10) == {"split": 3, "fused": True}
    cpgrad.set_als_plan([100] * 4, 10, 1)
    assert cpgrad.als_plan([100] * 4, 10) == 1
    for bad in (0, 4):
        with pytest.raises(cpgrad.CpgError):
            cpgrad.set_gradient_plan([100] * 4, 10, bad, False)
        with pytest.raises(cpgrad.CpgError):
            cpgrad.set_als_plan([100] * 4, 10, bad)
    with pytest.raises(cpgrad.CpgError) as e:
        cpgrad.set_gradient_plan([100] * 4, 10, 2, True, precision="bf16x6")
    assert e.value.status == cpgrad.CPG_ERR_UNSUPPORTED
    # the workspace of a gradient covers the recorded plan
    assert cpgrad.cpg_workspace_size([100] * 4, 10, "fp32", 0, cpgrad.CALL_GRADIENT_ALL) > 0
    cpgrad.autotune_clear()
    assert cpgrad.gradient_plan([100] * 4, 10) is None and cpgrad.als_plan([100] * 4, 10) is None
