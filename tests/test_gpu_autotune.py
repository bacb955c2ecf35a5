"""The measured plan choice of the all-mode gradient (cpg_autotune_gradient):
every candidate computes the same gradient (Algorithm 2 is exact for any
split, steps 4 and 7 fused or not), the recorded plan is one of them, and
later cp_gradient_all calls stay within the oracle tolerances."""
import numpy as np
import pytest

import cpsynth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as m
    yield m
    m.autotune_clear()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("I,R,prec", [([24, 20, 30, 17], 12, "fp32"), ([24, 20, 30, 17], 12, "bf16x3"),
                                      ([16, 12, 20, 8, 10], 6, "tf32x3"), ([40, 36, 28], 5, "bf16")])
def test_autotuned_plan_is_used_and_exact(cg, I, R, prec):
    y = cpsynth.random_tensor(I, seed=31)
    A = cpsynth.random_factors(I, R, seed=31)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    plan = cg.cp_gradient_autotune(Y, I, Ad, precision=prec, reps=2)
    N = len(I)
    assert 1 <= plan["split"] <= N - 1 and plan["ms"] > 0
    assert plan["candidates"] >= N - 1
    assert cg.gradient_plan(I, R, precision=prec) == {"split": plan["split"], "fused": plan["fused"]}
    if prec == "tf32x3":
        assert not plan["fused"]  # the split-TF32 kernel has no fused pass
    for _ in range(2):  # the recorded plan, twice
        G = cg.cp_gradient_all(Y, I, Ad, precision=prec)
        torch.cuda.synchronize()
        for n in range(N):
            assert _rel(G[n].double().cpu().numpy(), want[n]) <= TOL[prec], (plan, n)


def test_autotune_keeps_a_requested_split(cg):
    I, R = [14, 18, 11, 16], 7
    y = cpsynth.random_tensor(I, seed=33)
    A = cpsynth.random_factors(I, R, seed=33)
    Y = torch.from_numpy(y).cuda()
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    plan = cg.cp_gradient_autotune(Y, I, Ad, split=3, reps=1)
    assert plan["split"] == 3 and plan["candidates"] <= 2
    G = cg.cp_gradient_all(Y, I, Ad, split=3)
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for n in range(len(I)):
        assert _rel(G[n].double().cpu().numpy(), want[n]) <= 1e-5
