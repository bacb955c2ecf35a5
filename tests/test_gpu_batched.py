"""GPU checks of cp_als_batched: many independent tensors of mixed order,
shape and rank in one call give exactly the results of one cp_als_iter call
per tensor (same kernels, fixed summation orders), and match the FP64 oracle."""
import numpy as np
import pytest

import cpsynth
import oracle
from als_checks import sweep_backward_errors

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
    return torch.from_numpy(np.ascontiguousarray(a.T).astype(dtype)).cuda().t()


def mixed_batch(count, seed, dtype, orders=(2, 3, 4, 5)):
    """Members with N in {2..5}, I_n in [3, 24], R in [1, min(12, min I_n)]
    (so that every normal-equation matrix is positive definite), each a
    rank-R CP model plus 20 dB noise, and a seeded N(0,1) start."""
    rng = cpsynth.rng(seed, 99)
    out = []
    for b in range(count):
        N = int(rng.choice(orders))
        I = [int(v) for v in rng.integers(3, 25, size=N)]
        R = int(rng.integers(1, min(12, min(I)) + 1))
        out.append(cpsynth.make_problem(I, R, snr_db=20.0, seed=seed * 1000 + b, dtype=dtype))
    return out


@pytest.mark.parametrize("prec,count", [("fp32", 7), ("fp32", 40), ("fp64", 5), ("bf16x6", 6), ("tf32x3", 6)])
def test_batched_equals_separate_calls(cg, prec, count):
    dt = np.float64 if prec == "fp64" else np.float32
    probs = mixed_batch(count, seed=3 + count, dtype=dt)
    iters = 4
    Ys = [torch.from_numpy(p.y).cuda() for p in probs]
    A_b = [[dev_factor(a, dt) for a in p.init] for p in probs]
    A_s = [[a.clone() for a in A] for A in A_b]
    res_b = cg.cp_als_batched([(Y, p.I, A) for Y, p, A in zip(Ys, probs, A_b)], iters, precision=prec)
    res_s = [cg.cp_als_iter(Y, p.I, A, iters, precision=prec) for Y, p, A in zip(Ys, probs, A_s)]
    torch.cuda.synchronize()
    assert cg.cpg_device_status() == 0
    for b in range(count):
        for a1, a2 in zip(A_b[b], A_s[b]):
            assert torch.equal(a1, a2), b
        assert torch.equal(res_b[b][0], res_s[b][0]), b
        assert torch.equal(res_b[b][1], res_s[b][1]), b


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_batched_matches_oracle(cg, prec):
    """Each batched sweep, for every member: every mode's update against the
    oracle's normal equations (backward error 1e-5, tests/als_checks.py) and
    the fit against one oracle sweep from the same factors (1e-5).  A forward
    comparison of the factors would amplify the gradient's rounding by the
    normal equations' conditioning, which on the small members exceeds 1e-5
    even in FP32.  Orders >= 3: an order-2 member with R = min(I) is fitted
    exactly, where the cheap fit formula's cancellation (about sqrt(FP32
    epsilon)) would dominate the comparison."""
    probs = mixed_batch(5, seed=11, dtype=np.float32, orders=(3, 4, 5))
    Ys = [torch.from_numpy(p.y).cuda() for p in probs]
    A = [[a.astype(np.float32) for a in p.init] for p in probs]
    for sweep in range(3):
        A_b = [[dev_factor(a, np.float32) for a in Ab] for Ab in A]
        res = cg.cp_als_batched([(Y, p.I, Ad) for Y, p, Ad in zip(Ys, probs, A_b)], 1, precision=prec)
        torch.cuda.synchronize()
        for b, p in enumerate(probs):
            got = [a.double().cpu().numpy() for a in A_b[b]]
            y = p.y.astype(np.float64)
            errs = sweep_backward_errors(y, p.I, A[b], got)
            assert max(errs.values()) <= 1e-5, (sweep, b, errs)
            tr = oracle.cp_als(y, p.I, [a.astype(np.float64) for a in A[b]], iters=1)
            fit = float(res[b][1].cpu().numpy()[0])
            assert abs(fit - tr.fits[0]) <= 1e-5, (sweep, b, fit, tr.fits)
            A[b] = [g.astype(np.float32) for g in got]
    assert cg.cpg_device_status() == 0


def test_batched_is_ordered_on_the_caller_stream(cg):
    """Work enqueued on the caller's stream after the call sees the results."""
    probs = mixed_batch(20, seed=5, dtype=np.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Ys = [torch.from_numpy(p.y).cuda() for p in probs]
        A_b = [[dev_factor(a, np.float32) for a in p.init] for p in probs]
        res = cg.cp_als_batched([(Y, p.I, A) for Y, p, A in zip(Ys, probs, A_b)], 2, stream=s)
        snap = [A[0].clone() for A in A_b]  # ordered after the batch on s
    s.synchronize()
    for b in range(len(probs)):
        assert torch.equal(snap[b], A_b[b][0])


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_batched_graph_replay(cg, prec):
    """One cp_als_batched call captured in a CUDA graph (the pool streams are
    forked from and joined into the capturing stream) and replayed twice:
    bitwise the results of the same call made directly."""
    probs = mixed_batch(12, seed=19, dtype=np.float32)
    iters = 3
    Ys = [torch.from_numpy(p.y).cuda() for p in probs]
    A0 = [[dev_factor(a, np.float32) for a in p.init] for p in probs]
    A_ref = [[a.clone() for a in A] for A in A0]
    ref = cg.cp_als_batched([(Y, p.I, A) for Y, p, A in zip(Ys, probs, A_ref)], iters, precision=prec)
    torch.cuda.synchronize()
    # buffers the graph reads and writes, allocated before the capture
    A_g = [[a.clone() for a in A] for A in A0]
    lams = [torch.ones(p.R, dtype=torch.float64, device="cuda") for p in probs]
    fits = [torch.zeros(iters, dtype=torch.float64, device="cuda") for _ in probs]
    members = [(Y, p.I, A, lam, fit) for Y, p, A, lam, fit in zip(Ys, probs, A_g, lams, fits)]
    ws = cg.Workspace()
    cg.cp_als_batched(members, iters, precision=prec, workspace=ws)  # sizes the workspace, creates the pool
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for A, A_init in zip(A_g, A0):
            for a, a0 in zip(A, A_init):
                a.copy_(a0)
        cg.cp_als_batched(members, iters, precision=prec, workspace=ws)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for b in range(len(probs)):
            for a1, a2 in zip(A_g[b], A_ref[b]):
                assert torch.equal(a1, a2), b
            assert torch.equal(lams[b], ref[b][0]), b
            assert torch.equal(fits[b], ref[b][1]), b
    assert cg.cpg_device_status(ws) == 0


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_batched_runs_recorded_splits(cg, prec):
    """Members whose CP_ALS split was recorded (as cpg_autotune_als records
    it) run that split inside cp_als_batched: the same bits as cp_als_iter
    at that split, and the oracle's normal equations in that split's mode
    order (backward error, tests/als_checks.py)."""
    probs = [p for p in mixed_batch(12, seed=77, dtype=np.float32, orders=(3, 4, 5))][:6]
    splits = [len(p.I) - 1 if oracle.split_point(p.I) != len(p.I) - 1 else 1 for p in probs]
    cg.autotune_clear()
    for p, k in zip(probs, splits):
        cg.set_als_plan(p.I, p.R, k, precision=prec)
    try:
        Ys = [torch.from_numpy(p.y).cuda() for p in probs]
        A_b = [[dev_factor(a, np.float32) for a in p.init] for p in probs]
        A_s = [[a.clone() for a in A] for A in A_b]
        cg.cp_als_batched([(Y, p.I, A) for Y, p, A in zip(Ys, probs, A_b)], 1, precision=prec)
        for Y, p, A, k in zip(Ys, probs, A_s, splits):
            cg.cp_als_iter(Y, p.I, A, 1, precision=prec, split=k)
        torch.cuda.synchronize()
        assert cg.cpg_device_status() == 0
        for b, (p, k) in enumerate(zip(probs, splits)):
            assert all(torch.equal(a1, a2) for a1, a2 in zip(A_b[b], A_s[b])), b
            got = [a.double().cpu().numpy() for a in A_b[b]]
            errs = sweep_backward_errors(p.y, p.I, [a.astype(np.float32) for a in p.init], got,
                                         order=oracle.als_mode_order(p.I, k))
            assert max(errs.values()) <= 1e-5, (b, k, errs)
    finally:
        cg.autotune_clear()
