"""GPU parity of the gradient's consumers against the FP64 oracle: the cost
gradient of eq. 2.13 with its model term, the all-at-once first-order step of
eq. 2.15, and the multiplicative nonnegative updates of eq. 2.18 (all through
the C ABI).

Tolerances: the cost gradient's error is measured against the size of its
product term Y_(n) KR (the model term cancels much of it near a fit):
1e-5 for FP32 and the split BF16x3 product, 1e-12 for FP64.  Steps and NTF
sweeps: factors within 1e-5 (FP32) / 1e-10 (FP64) of the oracle's, relative
to the factor's norm."""
import numpy as np
import pytest

import cpsynth
import oracle

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


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a.T).astype(dt)).cuda().t()


@pytest.mark.parametrize("I,R,prec", [([24, 20, 30, 17], 12, "fp32"), ([30, 40, 50], 5, "fp64"),
                                      ([15, 15, 15, 15, 15], 10, "fp32"), ([40, 12, 8, 20], 8, "bf16x3"),
                                      ([9, 10, 11], 70, "fp32")])
def test_cost_gradient_matches_oracle(cg, I, R, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    p = cpsynth.make_problem(I, R, snr_db=10.0, seed=41, dtype=dt)
    Y = torch.from_numpy(p.y).cuda()
    A = [a.astype(dt).astype(np.float64) for a in p.init]
    G = cg.cp_gradient_full(Y, I, [dev(a, dt) for a in A], precision=prec)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 1e-5
    y = p.y.astype(np.float64)
    for n in range(len(I)):
        want = oracle.cp_gradient_full(y, I, A, n)
        scale = np.linalg.norm(oracle.cp_gradient(y, I, A, n))
        err = np.linalg.norm(G[n].double().cpu().numpy() - want) / scale
        assert err <= tol, (n, err)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gradient_step_matches_oracle(cg, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    I, R = [20, 24, 16, 18], 6
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=42, dtype=dt)
    y = p.y.astype(np.float64)
    A = [a.astype(dt).astype(np.float64) for a in p.init]
    # a step of about 1% of the factors' size along the gradient
    G0 = [oracle.cp_gradient_full(y, I, A, n) for n in range(len(I))]
    eta = 0.01 * sum(np.linalg.norm(a) for a in A) / sum(np.linalg.norm(g) for g in G0)
    Ad = [dev(a, dt) for a in A]
    Y = torch.from_numpy(p.y).cuda()
    G = cg.cp_gradient_step(Y, I, Ad, eta, precision=prec)
    torch.cuda.synchronize()
    A1, Gw = oracle.cp_gradient_step(y, I, A, eta)
    tol = 1e-10 if prec == "fp64" else 1e-5
    for n in range(len(I)):
        assert np.linalg.norm(Ad[n].double().cpu().numpy() - A1[n]) <= tol * np.linalg.norm(A1[n]), n
        scale = np.linalg.norm(oracle.cp_gradient(y, I, A, n))
        assert np.linalg.norm(G[n].double().cpu().numpy() - Gw[n]) <= tol * scale, n
    assert oracle.cp_cost(y, [a.double().cpu().numpy() for a in Ad]) < oracle.cp_cost(y, A)


def _nonneg(I, R, seed, noise, dt):
    rng = cpsynth.rng(seed, 7)
    A = [np.abs(rng.standard_normal((In, R))) + 0.1 for In in I]
    y = cpsynth.cp_model_vec(A)
    y = (y + noise * np.abs(rng.standard_normal(y.shape)) * np.std(y)).astype(dt)
    A0 = [(np.abs(rng.standard_normal((In, R))) + 0.1).astype(dt) for In in I]
    return y, A0


@pytest.mark.parametrize("I,R,prec,iters", [([20, 16, 24, 12], 5, "fp32", 4), ([30, 40, 50], 4, "fp64", 5),
                                            ([12, 10, 8, 9, 7], 3, "fp32", 3)])
def test_ntf_matches_oracle(cg, I, R, prec, iters):
    dt = np.float64 if prec == "fp64" else np.float32
    y, A0 = _nonneg(I, R, 43, 0.2, dt)
    Ad = [dev(a, dt) for a in A0]
    fit = cg.cp_ntf_iter(torch.from_numpy(y).cuda(), I, Ad, iters, precision=prec)
    torch.cuda.synchronize()
    tr = oracle.cp_ntf(y.astype(np.float64), I, [a.astype(np.float64) for a in A0], iters)
    tol = 1e-10 if prec == "fp64" else 1e-5
    for n in range(len(I)):
        got = Ad[n].double().cpu().numpy()
        assert np.all(got >= 0)
        assert np.linalg.norm(got - tr.A[n]) <= tol * np.linalg.norm(tr.A[n]), n
    f = fit.cpu().numpy()
    np.testing.assert_allclose(f, tr.fits, atol=tol)
    assert np.all(np.diff(f) >= -tol)  # multiplicative updates never raise the cost
    assert cg.cpg_device_status() == 0
