"""The two sources of the Khatri-Rao rows of the CUDA-core leading passes give
bitwise the same results.

When the tensor's rows are whole 16-byte units and its base is 16-byte
aligned, tiles arrive by TMA and W_R / W_L (eq. 3.10 / 3.9) are built once per
pass and copied with every tile.  A tensor whose first element sits 4 bytes
past a 16-byte boundary takes element copies, and every CTA then generates
its rows itself.  Both paths put the same tile and the same rows in shared
memory and run the same arithmetic in the same order, so their gradients and
ALS sweeps must agree bit for bit: this pins the built rows' layouts, padding,
per-stage slots and rank-group offsets to the per-CTA generation, which the
parity tests pin to the oracle."""
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
    return m


def dev_factor(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a.T).astype(dtype)).cuda()
    return t.t()


def two_copies(y):
    """The tensor at a 16-byte aligned address and at an address one element past one."""
    a = torch.from_numpy(y).cuda()
    buf = torch.empty(y.size + 4, dtype=a.dtype, device="cuda")
    b = buf[1:1 + y.size]  # one element (4 or 8 bytes) past the allocation's aligned start
    b.copy_(a)
    assert a.data_ptr() % 16 == 0 and b.data_ptr() % 16 != 0
    return a, b


CASES = [
    ([24, 20, 30, 17], 12, "fp32"),   # k=2, J=480: ragged row tile and column chunk, rank tile 12
    ([100, 100, 100], 20, "fp32"),    # k=1, J=100: step 7 with rank tile 24 (step 4 generates its rows)
    ([64, 64, 64, 4], 3, "fp32"),     # rank tile 4, 256-row tiles taller than J=64
    ([16, 16, 16, 16], 10, "fp32"),   # k=2, J=K=256
    ([40, 36, 28, 20], 16, "fp32"),   # k=2, J=1440, rank tile 16
    ([30, 40, 50], 5, "fp64"),        # FP64, J=30
    ([20, 22, 23], 20, "fp64"),       # FP64, two rank groups of 16
]


@pytest.mark.parametrize("I,R,prec", CASES)
def test_built_rows_match_per_cta_rows_gradient(cg, I, R, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    y = cpsynth.random_tensor(I, seed=21, dtype=dt)
    A = [dev_factor(a, dt) for a in cpsynth.random_factors(I, R, seed=21, dtype=dt)]
    ya, yb = two_copies(y)
    ws = cg.Workspace(torch.device("cuda"))
    Ga = [g.clone() for g in cg.cp_gradient_all(ya, I, A, workspace=ws, precision=prec)]
    Gb = cg.cp_gradient_all(yb, I, A, workspace=ws, precision=prec)
    torch.cuda.synchronize()
    for n, (a, b) in enumerate(zip(Ga, Gb)):
        assert torch.equal(a, b), f"mode {n}: max |diff| {float((a - b).abs().max())}"


@pytest.mark.parametrize("I,R", [([24, 20, 30, 17], 12), ([16, 16, 16, 16], 10)])
def test_built_rows_match_per_cta_rows_als(cg, I, R):
    y = cpsynth.random_tensor(I, seed=22, dtype=np.float32)
    A0 = [dev_factor(a, np.float32) for a in cpsynth.random_factors(I, R, seed=22, dtype=np.float32)]
    ya, yb = two_copies(y)
    ws = cg.Workspace(torch.device("cuda"))
    Aa = [a.clone() for a in A0]
    Ab = [a.clone() for a in A0]
    la, fa = cg.cp_als_iter(ya, I, Aa, 3, workspace=ws)
    lb, fb = cg.cp_als_iter(yb, I, Ab, 3, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(fa, fb) and torch.equal(la, lb)
    for a, b in zip(Aa, Ab):
        assert torch.equal(a, b)


class FixedWorkspace:
    """A workspace of exactly `nbytes` (the library's own helper grows to what a call asks for)."""

    def __new__(cls, cg, nbytes):
        class _Fixed(cg.Workspace):
            def get(self, want, stream_ptr):
                return super().get(nbytes, stream_ptr)
        return _Fixed(torch.device("cuda"))


def without_copy_bytes(cg, I, R, prec, k, call, J, K):
    """Workspace bytes of `call` less the pitched copy of Y (the last 256-byte aligned slot of the layout)."""
    full = cg.cpgrad.cpg_workspace_size(I, R, prec, k, call)
    esize = 8 if prec == "fp64" else 4
    q = 16 // esize
    copy = ((J + q - 1) // q * q) * K * esize
    return full - (copy + 255) // 256 * 256


# Tensors whose column pitch J is not a multiple of 16 bytes: with room in the
# workspace the library copies Y once with a padded pitch and every pass takes
# TMA tiles with built rows; without it, element copies and per-CTA rows.
PITCH_CASES = [
    ([15, 15, 15, 15, 15], 10, "fp32", 2),   # J = 225
    ([9, 11, 13, 7], 8, "fp32", 2),          # J = 99
    ([13, 7, 9, 11], 8, "fp64", 1),          # J = 13 (104-byte pitch)
]


@pytest.mark.parametrize("I,R,prec,k", PITCH_CASES)
def test_pitched_copy_matches_element_copies(cg, I, R, prec, k):
    dt = np.float64 if prec == "fp64" else np.float32
    y = cpsynth.random_tensor(I, seed=23, dtype=dt)
    A0 = [dev_factor(a, dt) for a in cpsynth.random_factors(I, R, seed=23, dtype=dt)]
    Y = torch.from_numpy(y).cuda()
    J = int(np.prod(I[:k]))
    K = int(np.prod(I[k:]))
    assert (J * y.itemsize) % 16 != 0
    big = cg.Workspace(torch.device("cuda"))

    def grad(ws):
        return [g.clone() for g in cg.cp_gradient_all(Y, I, A0, workspace=ws, precision=prec, split=k)]

    def als(ws):
        A = [a.clone() for a in A0]
        lam, fit = cg.cp_als_iter(Y, I, A, 3, workspace=ws, precision=prec, split=k)
        return A + [lam, fit]

    for call, run in ((cg.cpgrad.CALL_GRADIENT_ALL, grad), (cg.cpgrad.CALL_ALS, als)):
        small = FixedWorkspace(cg, without_copy_bytes(cg, I, R, prec, k, call, J, K))
        a = run(big)
        b = run(small)
        torch.cuda.synchronize()
        for x, z in zip(a, b):
            assert torch.equal(x, z), f"call {call}: max |diff| {float((x - z).abs().max())}"
