"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: relative Frobenius error per mode <= 1e-5 for the FP32 path and
the split BF16x3 / BF16x6 / TF32x3 products, 2e-2 for pure BF16, and
<= 1e-12 for the FP64 path (the bounds the method's target states for FP32
and a choice for FP64).  CP_ALS (FP32, TF32x3, BF16x6): fits within 1e-5,
factors and lambda after a sweep within 1e-5 relative; FP64 within 1e-9."""
import numpy as np
import pytest

import cpsynth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12, "bf16x3": 1e-5, "bf16x6": 1e-5, "tf32x3": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as m
    return m


def dev_factor(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a.T).astype(dtype)).cuda()  # (R, I) row-major = (I, R) column-major
    return t.t()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def inputs(I, R, prec, seed=1):
    dt = np.float64 if prec == "fp64" else np.float32
    y = cpsynth.random_tensor(I, seed=seed, dtype=dt)
    A = cpsynth.random_factors(I, R, seed=seed, dtype=dt)
    return y, A, dt


GRAD_CASES = [
    ([30, 40, 50], 5, "fp32"),          # k=1, J=30: element-wise copies
    ([37, 41, 29, 23], 10, "fp32"),     # k=1, ragged columns
    ([24, 20, 30, 17], 12, "fp32"),     # k=2, J=480: 16-byte copies, ragged row tile
    ([15, 15, 15, 15, 15], 10, "fp32"),  # k=2, J=225
    ([8, 8, 8, 8, 8, 8], 17, "fp32"),   # rank tile 24, row tile 64
    ([6, 7, 8, 9, 10], 33, "fp32"),     # rank tile 48, row tile 32
    ([12, 11, 10, 9], 64, "fp32"),
    ([9, 10, 11], 70, "fp32"),          # two rank groups
    ([20, 30, 40], 1, "fp32"),
    ([2, 3], 3, "fp32"),
    ([1, 5, 1], 2, "fp32"),
    ([300, 7], 4, "fp32"),              # I_1 > I_2: split clamped to 1
    ([5, 600], 8, "fp32"),
    ([4, 5, 3, 4, 3, 5, 4], 6, "fp32"),
    ([100, 100, 100], 20, "fp32"),      # two-pass route (partials of the fused pass too large)
    ([64, 64, 64, 4], 3, "fp32"),       # rank tile 4, row tile 256
    ([30, 40, 50], 5, "fp64"),
    ([13, 7, 9, 11], 8, "fp64"),
    ([21, 22, 23], 16, "fp64"),
    ([5, 6, 7], 20, "fp64"),            # two rank groups in FP64
    ([20, 22, 23], 20, "fp64"),         # two rank groups, J=20: TMA tiles with built Khatri-Rao rows
    # split-BF16 forms on the tensor cores (TMA boxes when J * 4 is a multiple
    # of 16, element copies otherwise)
    ([24, 20, 30, 17], 12, "bf16x3"),   # k=2, J=480: ragged row tile and column chunk
    ([100, 100, 100], 20, "bf16x3"),    # k=1, J=100, rank tile 32
    ([64, 64, 64, 4], 3, "bf16x3"),
    ([32, 16, 20, 24, 10], 10, "bf16x3"),
    ([12, 11, 10, 9], 64, "bf16x3"),    # rank tile 64 (J=132)
    ([9, 10, 11], 70, "bf16x3"),        # J=9: element copies, two rank groups
    ([15, 15, 15, 15, 15], 10, "bf16x3"),  # J=225: element copies
    ([7, 9, 11, 13], 20, "bf16"),       # J=63: element copies, pure BF16
    ([20, 12, 40, 36], 33, "bf16x3"),   # rank tile 64, R not a multiple of 16
    ([40, 36, 28, 20], 16, "bf16"),
    ([100, 100, 100], 10, "bf16"),
    # three BF16 limbs (six products)
    ([24, 20, 30, 17], 12, "bf16x6"),   # k=2, J=480: ragged row tile and column chunk
    ([100, 100, 100], 20, "bf16x6"),    # k=1, J=100, rank tile 32
    ([64, 64, 64, 4], 3, "bf16x6"),     # K=16384: many column chunks per CTA
    ([32, 16, 20, 24, 10], 10, "bf16x6"),
    ([12, 11, 10, 9], 64, "bf16x6"),    # rank tile 64
    ([9, 10, 11], 70, "bf16x6"),        # J=9: element loads, two rank groups
    ([15, 15, 15, 15, 15], 10, "bf16x6"),  # J=225: element loads
    ([20, 12, 40, 36], 33, "bf16x6"),   # rank tile 64, R not a multiple of 16
    ([10, 12, 14], 130, "bf16x6"),      # three rank groups: the B tiles rebuilt per group
    ([16, 8, 24, 6], 200, "bf16x3"),    # four rank groups, the last of 8 ranks
    # split-TF32 products on the tensor cores (one side per pass; 128 x 64
    # step-4 tiles, 64 x 128 step-7 tiles)
    ([24, 20, 30, 17], 12, "tf32x3"),   # k=2, J=480: TMA boxes, ragged row tile and column chunk
    ([100, 100, 100], 20, "tf32x3"),    # k=1, J=100, rank tile 32
    ([64, 64, 64, 4], 3, "tf32x3"),     # k=1, J=64, K=16384: many column chunks
    ([12, 11, 10, 9], 64, "tf32x3"),    # rank tile 64
    ([9, 10, 11], 70, "tf32x3"),        # J=9: element copies, two rank groups
    ([15, 15, 15, 15, 15], 10, "tf32x3"),  # J=225: element copies
    ([20, 12, 40, 36], 33, "tf32x3"),   # rank tile 64, R not a multiple of 16
]


@pytest.mark.parametrize("I,R,prec", GRAD_CASES)
def test_gradient_all(cg, I, R, prec):
    y, A, dt = inputs(I, R, prec)
    Y = torch.from_numpy(y).cuda()
    Ad = [dev_factor(a, dt) for a in A]
    G = cg.cp_gradient_all(Y, I, Ad, precision=prec)
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for n in range(len(I)):
        e = rel(G[n].double().cpu().numpy(), want[n])
        assert e <= TOL[prec], f"mode {n}: rel err {e:.3e}"


@pytest.mark.parametrize("split", [1, 2, 3])
def test_gradient_all_split_override(cg, split):
    I, R = [14, 18, 11, 16], 7
    y, A, dt = inputs(I, R, "fp32", seed=3)
    Y = torch.from_numpy(y).cuda()
    G = cg.cp_gradient_all(Y, I, [dev_factor(a, dt) for a in A], split=split)
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for n in range(len(I)):
        assert rel(G[n].double().cpu().numpy(), want[n]) <= 1e-5


@pytest.mark.parametrize("I,R,prec", [([30, 40, 50], 5, "fp32"), ([11, 9, 13, 7, 5], 9, "fp32"),
                                      ([200, 3, 4], 6, "fp32"), ([3, 4, 200], 6, "fp32"),
                                      ([13, 7, 9, 11], 8, "fp64"), ([40, 12, 8, 20], 8, "bf16x3"),
                                      ([4, 8, 300], 6, "bf16x3"), ([40, 12, 8, 20], 8, "tf32x3"),
                                      ([40, 12, 8, 20], 8, "bf16x6"), ([4, 8, 300], 6, "bf16x6"),
                                      ([4, 8, 300], 6, "tf32x3")])
def test_gradient_mode(cg, I, R, prec):
    y, A, dt = inputs(I, R, prec, seed=5)
    Y = torch.from_numpy(y).cuda()
    Ad = [dev_factor(a, dt) for a in A]
    for n in range(len(I)):
        Gn = cg.cp_gradient_mode(Y, I, Ad, n, precision=prec)
        torch.cuda.synchronize()
        want = oracle.cp_gradient(y.astype(np.float64), I, A, n)
        assert rel(Gn.double().cpu().numpy(), want) <= TOL[prec], f"mode {n}"


def test_gradient_exact_cp_closed_form(cg):
    """eq. 2.13 with E = 0 on the device: Y = [[A]] gives G^(n) = A^(n) (Hadamard of the other Grams)."""
    I, R = [20, 24, 28, 16], 5
    A = cpsynth.gaussian_factors(I, R, seed=8)
    A = [a.astype(np.float32).astype(np.float64) for a in A]
    y = cpsynth.cp_model_vec(A).astype(np.float32)
    G = cg.cp_gradient_all(torch.from_numpy(y).cuda(), I, [dev_factor(a, np.float32) for a in A])
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for n in range(len(I)):
        assert rel(G[n].double().cpu().numpy(), want[n]) <= 1e-5


def test_gradient_deterministic(cg):
    I, R = [24, 20, 30, 17], 12
    y, A, dt = inputs(I, R, "fp32", seed=9)
    Y = torch.from_numpy(y).cuda()
    Ad = [dev_factor(a, dt) for a in A]
    G1 = [g.clone() for g in cg.cp_gradient_all(Y, I, Ad)]
    G2 = cg.cp_gradient_all(Y, I, Ad)
    torch.cuda.synchronize()
    for a, b in zip(G1, G2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("R", [10, 20])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "bf16x6", "bf16"])
def test_precision_study_7d(cg, R, prec):
    """The 7-D collinear workload's recipe (factor columns with pairwise
    cosine 0.5, 30 dB noise) at I = 7 per mode: per-mode relative Frobenius
    error of every precision against the FP64 oracle.  J = 343 rows per
    column are not 16-byte multiples, so the tensor-core forms take the
    element-copy path."""
    p = cpsynth.make_problem([7] * 7, R, snr_db=30.0, seed=7, dtype=np.float32, collinearity=0.5)
    Y = torch.from_numpy(p.y).cuda()
    Ad = [dev_factor(a, np.float32) for a in p.factors]
    G = cg.cp_gradient_all(Y, p.I, Ad, precision=prec)
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(p.y.astype(np.float64), p.I, p.factors)
    errs = [rel(G[n].double().cpu().numpy(), want[n]) for n in range(7)]
    assert max(errs) <= TOL[prec], errs
    if prec == "bf16":
        # One BF16 limb carries 8 significant bits: an error at FP32 level
        # would mean the call did not run the BF16 products.
        assert min(errs) > 1e-4, errs


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6", "tf32x3"])
def test_gradient_full_size_sampled(cg, prec):
    """The 4-D 100^4, R = 10 workload in the benchmark's launch configuration;
    sampled entries g_r^(n)[i] checked one by one with the oracle (eq. 3.2)."""
    p = cpsynth.workload("cp4d_100_r10_fp32")
    I, R = p.I, p.R
    Y = torch.from_numpy(p.y).cuda()
    Ad = [dev_factor(a, np.float32) for a in p.init]
    G = [g.double().cpu().numpy() for g in cg.cp_gradient_all(Y, I, Ad, precision=prec)]
    # every entry against the oracle's explicit unfolding x Khatri-Rao product
    want = oracle.cp_gradient_all(p.y, I, p.init)
    for n in range(len(I)):
        assert rel(G[n], want[n]) <= 1e-5, n
    # and a few entries one by one from the elementwise sum (eq. 3.2)
    rng = np.random.default_rng(0)
    for n in range(len(I)):
        for _ in range(3):
            i, r = int(rng.integers(I[n])), int(rng.integers(R))
            w = oracle.cp_gradient_entry(p.y, I, p.init, n, i, r)
            assert abs(want[n][i, r] - w) <= 1e-9 * max(1.0, abs(w))
    if prec == "bf16x3":
        return  # gradient-only precision
    # one ALS sweep from the same start: fit against the oracle's fit
    Ad = [dev_factor(a, np.float32) for a in p.init]
    lam, fit = cg.cp_als_iter(Y, I, Ad, 1, precision=prec)
    torch.cuda.synchronize()
    tr = oracle.cp_als(p.y, I, p.init, iters=1)
    assert abs(fit.cpu().numpy()[0] - tr.fits[0]) <= 1e-5


@pytest.mark.parametrize("I,R,prec,iters", [([30, 40, 50], 5, "fp64", 10), ([24, 20, 30, 17], 6, "fp32", 6),
                                            ([12, 10, 8, 9, 7], 4, "fp32", 5), ([40, 30], 3, "fp32", 8),
                                            ([24, 20, 30, 17], 6, "bf16x6", 6), ([40, 36, 28], 5, "bf16x6", 5),
                                            ([24, 20, 30, 17], 6, "tf32x3", 6), ([40, 36, 28], 5, "tf32x3", 5)])
def test_als_matches_oracle(cg, I, R, prec, iters):
    dt = np.float64 if prec == "fp64" else np.float32
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=11, dtype=dt)
    Y = torch.from_numpy(p.y).cuda()
    Ad = [dev_factor(a, dt) for a in p.init]
    lam, fit = cg.cp_als_iter(Y, I, Ad, iters, precision=prec)
    torch.cuda.synchronize()
    tr = oracle.cp_als(p.y.astype(np.float64), I, p.init, iters=iters)
    ftol = 1e-9 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(fit.cpu().numpy(), tr.fits, atol=ftol)
    if prec == "fp64":
        for n in range(len(I)):
            assert rel(Ad[n].cpu().numpy(), tr.A[n]) <= 1e-9
        np.testing.assert_allclose(lam.cpu().numpy(), tr.lam, rtol=1e-9)
    assert cg.cpg_device_status() == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x6"])
def test_als_one_sweep_factors(cg, prec):
    """Per-sweep parity from identical factors."""
    I, R = [24, 20, 30, 17], 6
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=12, dtype=np.float32)
    Ad = [dev_factor(a, np.float32) for a in p.init]
    lam, fit = cg.cp_als_iter(torch.from_numpy(p.y).cuda(), I, Ad, 1, precision=prec)
    torch.cuda.synchronize()
    tr = oracle.cp_als(p.y.astype(np.float64), I, p.init, iters=1)
    tol = 1e-5
    for n in range(len(I)):
        assert rel(Ad[n].double().cpu().numpy(), tr.A[n]) <= tol, n
    np.testing.assert_allclose(lam.cpu().numpy(), tr.lam, rtol=tol)


def test_als_noiseless_fit_to_one(cg):
    I, R = [16, 18, 14, 12], 3
    A = cpsynth.gaussian_factors(I, R, seed=4)
    y = cpsynth.cp_model_vec(A).astype(np.float64)
    A0 = cpsynth.gaussian_factors(I, R, seed=6)
    Ad = [dev_factor(a, np.float64) for a in A0]
    lam, fit = cg.cp_als_iter(torch.from_numpy(y).cuda(), I, Ad, 100, precision="fp64")
    torch.cuda.synchronize()
    # The cheap fit cancels O(||Y||^2) terms, so in FP64 it resolves a misfit
    # only down to about sqrt(eps) ~ 1.5e-8; the explicit fit has no such floor.
    assert fit.cpu().numpy()[-1] > 1 - 1e-7
    A = [a.cpu().numpy() for a in Ad]
    assert oracle.cp_fit_direct(y, A, lam.cpu().numpy()) > 1 - 1e-10


def test_als_singular_status(cg):
    """A zero column makes V singular for every mode but one: the first
    update that sees it reports CPG_ERR_SINGULAR and leaves its factor."""
    I, R = [10, 12, 14], 3
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=13, dtype=np.float32)
    A0 = [a.copy() for a in p.init]
    A0[2][:, 0] = 0.0
    Ad = [dev_factor(a, np.float32) for a in A0]
    before = Ad[0].clone()
    cg.cpg_device_status()  # clear
    cg.cp_als_iter(torch.from_numpy(p.y).cuda(), I, Ad, 1)
    assert cg.cpg_device_status() == 4
    assert torch.equal(Ad[0], before)
    assert cg.cpg_device_status() == 0


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_sweeps_refuse_gradient_only_precisions(cg, prec):
    """One or two BF16 limbs are gradient-only: CP_ALS returns
    CPG_ERR_UNSUPPORTED before launching anything."""
    I, R = [12, 10, 8], 3
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=14, dtype=np.float32)
    Ad = [dev_factor(a, np.float32) for a in p.init]
    with pytest.raises(cg.CpgError) as e:
        cg.cp_als_iter(torch.from_numpy(p.y).cuda(), I, Ad, 1, precision=prec)
    assert e.value.status == cg.CPG_ERR_UNSUPPORTED
