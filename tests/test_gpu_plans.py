"""Every plan of the all-mode gradient against the FP64 oracle.

The gradient autotuner (cpg_autotune_gradient) runs whichever plan times
fastest, one fused pass (Algorithm 2 steps 4 and 7 from one read of Y) or
two passes, at any split k; the planner alone fuses only some cases.  Each
plan is pinned here with cpg_gradient_plan_set, then run by cp_gradient_all
and compared with the oracle at the precision's tolerance."""
import numpy as np
import pytest

import cpsynth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16x6": 1e-5, "tf32x3": 1e-5, "bf16": 2e-2}
FUSED = {"fp32": True, "bf16x3": True, "bf16": True, "bf16x6": False, "tf32x3": False}


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as m
    yield m
    m.autotune_clear()


CASES = [
    ([8, 9, 10, 11], 4, "fp32"),         # rank tile 4
    ([24, 20, 30, 17], 12, "fp32"),      # rank tile 12, ragged tiles
    ([15, 12, 10, 8, 6], 20, "fp32"),    # rank tile 24
    ([20, 16, 12, 10], 32, "fp32"),      # rank tile 32
    ([24, 20, 30, 17], 12, "bf16x3"),
    ([20, 16, 12, 10], 32, "bf16x3"),    # rank tile 32, the widest fused tile
    ([40, 36, 28, 20], 16, "bf16"),
    ([24, 20, 30, 17], 12, "bf16x6"),
    ([24, 20, 30, 17], 12, "tf32x3"),
]


@pytest.mark.parametrize("I,R,prec", CASES)
def test_every_plan_matches_oracle(cg, I, R, prec):
    y = cpsynth.random_tensor(I, seed=51, dtype=np.float32)
    A = [a.astype(np.float32) for a in cpsynth.random_factors(I, R, seed=52)]
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    Y = torch.from_numpy(y).cuda()
    Ad = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t() for a in A]
    ran = 0
    for k in range(1, len(I)):
        for fused in ([False, True] if FUSED[prec] else [False]):
            cg.set_gradient_plan(I, R, k, fused, precision=prec)
            assert cg.gradient_plan(I, R, prec) == {"split": k, "fused": fused}
            G = cg.cp_gradient_all(Y, I, Ad, precision=prec)
            torch.cuda.synchronize()
            errs = [float(np.linalg.norm(G[n].double().cpu().numpy() - want[n]) / np.linalg.norm(want[n]))
                    for n in range(len(I))]
            assert max(errs) <= TOL[prec], (k, fused, errs)
            ran += 1
    assert cg.cpg_device_status() == 0
    cg.autotune_clear()
    assert ran >= len(I) - 1
