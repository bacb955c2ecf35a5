"""The CP_ALS split autotuner on the GPU (Section 4 with the sweep started at
a measured split k instead of n*).

- Every candidate split runs sweeps that match the oracle's sweep with the
  same mode order (k-1, ..., 0, k, ..., N-1): per-mode backward error of the
  factors in the oracle's normal equations, and the fit, both at 1e-5.
- The autotuner leaves the caller's factors and lambda bit-for-bit as they
  were, records its split, and a later sweep with split 0 runs that split
  (the same bits as a sweep that requests it)."""
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


def dev_factor(a):
    return torch.from_numpy(np.ascontiguousarray(a.T).astype(np.float32)).cuda().t()


CASES = [([12, 9, 10, 8, 11], 5), ([40, 36, 44], 7)]


@pytest.mark.parametrize("I,R", CASES)
@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_every_candidate_split_matches_oracle(cg, I, R, prec):
    y = cpsynth.random_tensor(I, seed=31, dtype=np.float32)
    A = cpsynth.random_factors(I, R, seed=32, dtype=np.float32)
    Y = torch.from_numpy(y).cuda()
    cands = cg.als_candidates(I, R)
    assert len(cands) >= 2, cands  # more than n* is exercised
    for k in cands:
        Ad = [dev_factor(a) for a in A]
        lam, fit = cg.cp_als_iter(Y, I, Ad, 1, precision=prec, split=k)
        torch.cuda.synchronize()
        got = [a.double().cpu().numpy() for a in Ad]
        order = oracle.als_mode_order(I, k)
        errs = sweep_backward_errors(y, I, A, got, order=order)
        assert max(errs.values()) <= 1e-5, (k, errs)
        tr = oracle.cp_als(y, I, [a.astype(np.float64) for a in A], iters=1, order=order)
        assert abs(float(fit.cpu().numpy()[0]) - tr.fits[0]) <= 1e-5, k


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_autotune_keeps_inputs_and_records_split(cg, prec):
    I, R = CASES[0]
    y = cpsynth.random_tensor(I, seed=33, dtype=np.float32)
    A = cpsynth.random_factors(I, R, seed=34, dtype=np.float32)
    Y = torch.from_numpy(y).cuda()
    Ad = [dev_factor(a) for a in A]
    lam = torch.linspace(1.0, 2.0, R, dtype=torch.float64, device="cuda")
    A_in = [a.clone() for a in Ad]
    lam_in = lam.clone()
    cg.autotune_clear()
    plan = cg.cp_als_autotune(Y, I, Ad, lam, precision=prec, reps=2)
    torch.cuda.synchronize()
    assert plan["split"] in cg.als_candidates(I, R)
    assert plan["candidates"] == len(cg.als_candidates(I, R)) and plan["ms"] > 0
    assert all(torch.equal(a, b) for a, b in zip(Ad, A_in))
    assert torch.equal(lam, lam_in)
    assert cg.als_plan(I, R, prec) == plan["split"]
    # split 0 now runs the recorded split
    A1 = [a.clone() for a in A_in]
    A2 = [a.clone() for a in A_in]
    _, f1 = cg.cp_als_iter(Y, I, A1, 3, precision=prec)
    _, f2 = cg.cp_als_iter(Y, I, A2, 3, precision=prec, split=plan["split"])
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(A1, A2))
    assert torch.equal(f1, f2)
    assert cg.cpg_device_status() == 0
    cg.autotune_clear()
    assert cg.als_plan(I, R, prec) is None
