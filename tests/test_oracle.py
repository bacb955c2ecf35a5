"""Pins for the FP64 oracle against facts fixed by the paper and by algebra,
none of which re-types the oracle's own unfold-and-multiply code.

* brute force of eq. 3.2 over every multi-index (ivec written out per eq. 2.1);
* the hand-worked integer example in tests/golden/;
* closed form of eq. 2.13 with E = 0 for an exact CP tensor;
* the invariant sum_i a_r^(n)[i] g_r^(n)[i] = Y x {a_r} for all n (eq. 2.6);
* N = 2: G^(1) = Y A^(2), G^(2) = Y^T A^(1);
* ALS (eq. 2.14): Eckart-Young on matrices, fit -> 1 on noiseless CP tensors,
  monotone cost, cheap fit formula = explicit fit;
* the cost gradient of eq. 2.13 (both terms) against central differences of
  D (eq. 2.12) summed entry by entry, and zero at an exact factorisation; a
  small first-order step (eq. 2.15) lowers D by 2 eta ||G||^2 to first order;
* multiplicative NTF (eq. 2.18): fixed point at an exact nonnegative
  factorisation, non-increasing D, nonnegative factors, cheap fit = explicit;
* the normal-equation solve of eq. 2.14 with a singular V (two equal factor
  columns): the result solves A V = G exactly when G is consistent and its
  rows lie in the range of V, which together make it G V^dagger.
"""
import itertools
import json
import os

import numpy as np
import pytest

import cpsynth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ivec(idx, I):
    """eq. 2.1, 0-based: i = i_1 + sum_n i_n * prod_{j<n} I_j."""
    lin, stride = 0, 1
    for i, n in zip(idx, I):
        lin += i * stride
        stride *= n
    return lin


def brute_gradient(y, I, A, n):
    """eq. 3.2 evaluated term by term in pure Python."""
    R = A[0].shape[1]
    G = np.zeros((I[n], R))
    for idx in itertools.product(*[range(v) for v in I]):
        yv = float(y[ivec(idx, I)])
        for r in range(R):
            p = yv
            for m, im in enumerate(idx):
                if m != n:
                    p *= A[m][im, r]
            G[idx[n], r] += p
    return G


def multi_tvp(y, I, A, r):
    """Y x_1 a^(1) x_2 ... x_N a^(N) (eq. 2.6) by contracting one mode at a time."""
    T = np.asarray(y, dtype=np.float64).reshape(I, order="F")
    for m in range(len(I)):
        T = np.tensordot(T, A[m][:, r], axes=([0], [0]))
    return float(T)


SHAPES = [
    ([3, 2], 1), ([2, 5], 3), ([1, 4], 2), ([3, 1, 2], 2), ([2, 3, 5], 3),
    ([5, 2, 3], 1), ([2, 2, 3, 2], 2), ([3, 1, 2, 5], 3), ([2, 3, 2, 2, 3], 2),
    ([1, 2, 1, 3, 2], 1),
]


@pytest.mark.parametrize("I,R", SHAPES)
def test_gradient_matches_bruteforce(I, R):
    g = cpsynth.rng(7, len(I), R)
    y = g.standard_normal(int(np.prod(I)))
    A = [g.standard_normal((v, R)) for v in I]
    for n in range(len(I)):
        Gb = brute_gradient(y, I, A, n)
        Go = oracle.cp_gradient(y, I, A, n)
        np.testing.assert_allclose(Go, Gb, rtol=1e-12, atol=1e-12)
        for i in range(I[n]):
            for r in range(R):
                assert oracle.cp_gradient_entry(y, I, A, n, i, r) == pytest.approx(Gb[i, r], rel=1e-12, abs=1e-12)
        # the batched form (slices formed once, FP32 input as the large tests pass it)
        pairs = [(i, r) for i in range(I[n]) for r in range(R)]
        got = oracle.cp_gradient_entries(y, I, A, n, pairs)
        np.testing.assert_allclose(got, [Gb[i, r] for i, r in pairs], rtol=1e-12, atol=1e-12)
        y32 = y.astype(np.float32)
        got32 = oracle.cp_gradient_entries(y32, I, A, n, pairs[::-1])
        want32 = brute_gradient(y32.astype(np.float64), I, A, n)
        np.testing.assert_allclose(got32, [want32[i, r] for i, r in pairs[::-1]], rtol=1e-12, atol=1e-12)


def test_golden_worked_example():
    with open(os.path.join(GOLDEN, "worked_example_3d.json")) as f:
        ex = json.load(f)
    I = ex["I"]
    y = np.array(ex["vecY"], dtype=np.float64)
    A = [np.array(a, dtype=np.float64) for a in ex["A"]]
    for n in range(len(I)):
        G = oracle.cp_gradient(y, I, A, n)
        np.testing.assert_array_equal(G, np.array(ex["G"][n], dtype=np.float64))
        np.testing.assert_array_equal(np.sum(A[n] * G, axis=0), np.array(ex["inner"], dtype=np.float64))


@pytest.mark.parametrize("I,R", [([4, 5, 6], 3), ([3, 4, 2, 5], 4), ([2, 3, 4, 3, 2], 2), ([6, 7], 5)])
def test_closed_form_exact_cp(I, R):
    """eq. 2.13 with E = 0: Y_(n) KR = A^(n) (Hadamard_{m != n} A^(m)T A^(m))."""
    A = cpsynth.gaussian_factors(I, R, seed=11)
    y = cpsynth.cp_model_vec(A)
    for n in range(len(I)):
        V = np.ones((R, R))
        for m in range(len(I)):
            if m != n:
                V *= A[m].T @ A[m]
        want = A[n] @ V
        got = oracle.cp_gradient(y, I, A, n)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("I,R", [([5, 4, 3], 3), ([3, 3, 3, 3], 2), ([2, 5, 3, 2, 2], 4)])
def test_invariant_inner_product(I, R):
    g = cpsynth.rng(3, len(I))
    y = g.standard_normal(int(np.prod(I)))
    A = [g.standard_normal((v, R)) for v in I]
    want = np.array([multi_tvp(y, I, A, r) for r in range(R)])
    for n in range(len(I)):
        G = oracle.cp_gradient(y, I, A, n)
        np.testing.assert_allclose(np.sum(A[n] * G, axis=0), want, rtol=1e-11, atol=1e-11)


def test_matrix_case():
    g = cpsynth.rng(5)
    I, R = [7, 9], 4
    y = g.standard_normal(63)
    A = [g.standard_normal((v, R)) for v in I]
    Y = y.reshape(I, order="F")
    np.testing.assert_allclose(oracle.cp_gradient(y, I, A, 0), Y @ A[1], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.cp_gradient(y, I, A, 1), Y.T @ A[0], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("I,k", [([100] * 4, 2), ([60] * 5, 2), ([15] * 7, 3), ([30, 40, 50], 1),
                                 ([100, 2], 1), ([2, 100], 1), ([2, 2], 1), ([1, 1, 1], 2),
                                 ([3, 4, 5, 6, 7], 2), ([10, 10, 10, 10, 10, 10, 10], 3)])
def test_split_point(I, k):
    assert oracle.split_point(I) == k


def test_mode_order():
    assert oracle.als_mode_order([100] * 4) == [1, 0, 2, 3]
    assert oracle.als_mode_order([15] * 7) == [2, 1, 0, 3, 4, 5, 6]
    assert oracle.als_mode_order([30, 40, 50]) == [0, 1, 2]


def test_solve_normal_singular_is_minimum_norm_solution():
    """A singular V, as when two columns of a factor coincide, sends the
    oracle's solve of eq. 2.14 to its eigen branch.  For G = X V (a
    consistent system) the Moore-Penrose solution G V^dagger is the unique A
    with A V = G whose rows lie in range(V): check both properties, plus a
    rank-one V built from equal columns, without forming a pseudo-inverse."""
    from oracle.cp_oracle import _solve_normal
    g = cpsynth.rng(41)
    R = 6
    B = g.standard_normal((R, 4))
    V = B @ B.T                                   # PSD, rank 4
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(V)
    X = g.standard_normal((9, R))
    G = X @ V
    A = _solve_normal(G, V)
    assert np.linalg.norm(A @ V - G) <= 1e-10 * np.linalg.norm(G)
    w, Q = np.linalg.eigh(V)
    null = Q[:, w < 1e-9 * w.max()]               # basis of V's null space
    assert null.shape[1] == 2
    assert np.linalg.norm(A @ null) <= 1e-10 * np.linalg.norm(A)
    # any other solution differs by a null-space term and is longer
    other = A + g.standard_normal((9, 2)) @ null.T
    assert np.linalg.norm(other @ V - G) <= 1e-10 * np.linalg.norm(G)
    assert np.linalg.norm(other) > np.linalg.norm(A)
    # equal columns: a^(m) columns 0 and 1 coincide in every other mode, so
    # V = Hadamard of the other Grams has equal rows/columns 0 and 1
    a = g.standard_normal((7, 3))
    a[:, 1] = a[:, 0]
    V2 = (a.T @ a) * (a.T @ a)
    G2 = g.standard_normal((5, 3)) @ V2
    A2 = _solve_normal(G2, V2)
    assert np.linalg.norm(A2 @ V2 - G2) <= 1e-10 * np.linalg.norm(G2)
    assert np.allclose(A2[:, 0], A2[:, 1], atol=1e-12 * np.abs(A2).max())  # no null-space component


def test_als_eckart_young():
    """N = 2: ALS on a matrix converges to its best rank-R approximation, whose
    residual is given by the trailing singular values."""
    g = cpsynth.rng(21)
    U, _ = np.linalg.qr(g.standard_normal((12, 12)))
    V, _ = np.linalg.qr(g.standard_normal((9, 9)))
    s = np.array([9.0, 7.0, 5.0, 3.0, 1.0, 0.5, 0.3, 0.2, 0.1])
    Y = U[:, :9] @ np.diag(s) @ V.T
    y = np.reshape(Y, -1, order="F")
    R = 3
    A0 = [g.standard_normal((12, R)), g.standard_normal((9, R))]
    tr = oracle.cp_als(y, [12, 9], A0, iters=200, direct_fit=True)
    want = 1.0 - np.sqrt(np.sum(s[R:] ** 2)) / np.sqrt(np.sum(s ** 2))
    assert tr.fits[-1] == pytest.approx(want, abs=1e-9)
    assert tr.fits_direct[-1] == pytest.approx(want, abs=1e-9)


def test_als_noiseless_fit_to_one_and_monotone():
    I, R = [8, 9, 7, 6], 3
    A = cpsynth.gaussian_factors(I, R, seed=4)
    y = cpsynth.cp_model_vec(A)
    # Starts 6 and 7 converge; start 5 sits in a swamp (a slow-progress stretch
    # that ALS is known for, end of Section 5) and is only checked for monotonicity.
    for seed, converges in ((6, True), (7, True), (5, False)):
        A0 = cpsynth.gaussian_factors(I, R, seed=seed)
        tr = oracle.cp_als(y, I, A0, iters=150, direct_fit=True)
        if converges:
            # the cheap fit bottoms out near sqrt(eps) (cancellation); the explicit one does not
            assert tr.fits[-1] > 1 - 1e-7
            assert tr.fits_direct[-1] > 1 - 1e-10
        d = np.array(tr.fits_direct)
        assert np.all(np.diff(d) >= -1e-12)
        np.testing.assert_allclose(tr.fits, tr.fits_direct, atol=1e-9)
        for n in range(len(I)):
            np.testing.assert_allclose(np.linalg.norm(tr.A[n], axis=0), 1.0, rtol=1e-12)


def test_als_cheap_fit_equals_direct_noisy():
    p = cpsynth.make_problem([6, 7, 8], 4, snr_db=10.0, seed=9, dtype=np.float64)
    tr = oracle.cp_als(p.y, p.I, p.init, iters=8, direct_fit=True)
    np.testing.assert_allclose(tr.fits, tr.fits_direct, rtol=1e-10, atol=1e-12)
    assert np.all(np.diff(tr.fits_direct) >= -1e-12)


def test_als_rank_one_is_power_iteration_on_matrix():
    """R = 1 on a matrix: ALS is the power method, so the model is the top
    singular triplet sigma_1 u v^T."""
    g = cpsynth.rng(33)
    Y = g.standard_normal((10, 8))
    y = np.reshape(Y, -1, order="F")
    tr = oracle.cp_als(y, [10, 8], [g.standard_normal((10, 1)), g.standard_normal((8, 1))], iters=300)
    s = np.linalg.svd(Y, compute_uv=False)
    assert tr.lam[0] == pytest.approx(s[0], rel=1e-9)


def test_cp_full_layout():
    """cp_full and the synthetic generator agree on the layout of eq. 2.1."""
    I, R = [3, 4, 2], 2
    A = cpsynth.gaussian_factors(I, R, seed=2)
    y = oracle.cp_full(A)
    for idx in itertools.product(*[range(v) for v in I]):
        want = sum(np.prod([A[m][idx[m], r] for m in range(3)]) for r in range(R))
        assert y[ivec(idx, I)] == pytest.approx(want, rel=1e-12, abs=1e-14)
    np.testing.assert_allclose(cpsynth.cp_model_vec(A), y, rtol=1e-12, atol=1e-14)


# ---- consumers of the gradient: eq. 2.13 (model term), eq. 2.15, eq. 2.18 -------------
def brute_cost(y, I, A):
    """D = ||Y - Yhat||^2 (eq. 2.12) with Yhat entry by entry from eq. 2.7."""
    R = A[0].shape[1]
    D = 0.0
    for idx in itertools.product(*[range(v) for v in I]):
        yhat = sum(np.prod([A[m][idx[m], r] for m in range(len(I))]) for r in range(R))
        D += (float(y[ivec(idx, I)]) - yhat) ** 2
    return D


@pytest.mark.parametrize("I,R", [([3, 4, 2], 2), ([2, 3, 2, 3], 3), ([4, 3], 2)])
def test_full_gradient_is_minus_half_cost_derivative(I, R):
    """Central differences of D (eq. 2.12, summed entry by entry) give
    dD/dA^(n) = -2 G^(n) with G^(n) of eq. 2.13 (both terms)."""
    rng = np.random.default_rng(5)
    y = rng.standard_normal(int(np.prod(I)))
    A = [rng.standard_normal((In, R)) for In in I]
    h = 1e-5
    for n in range(len(I)):
        G = oracle.cp_gradient_full(y, I, A, n)
        for i in range(I[n]):
            for r in range(R):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[n][i, r] += h
                Am[n][i, r] -= h
                fd = (brute_cost(y, I, Ap) - brute_cost(y, I, Am)) / (2 * h)
                assert abs(fd - (-2.0 * G[i, r])) <= 1e-6 * max(1.0, abs(fd)), (n, i, r, fd, G[i, r])
    assert abs(oracle.cp_cost(y, A) - brute_cost(y, I, A)) <= 1e-9 * brute_cost(y, I, A)


@pytest.mark.parametrize("I,R", [([5, 6, 7], 3), ([4, 3, 5, 2], 2)])
def test_full_gradient_vanishes_at_exact_factorisation(I, R):
    A = cpsynth.gaussian_factors(I, R, seed=14)
    y = cpsynth.cp_model_vec(A)
    for n in range(len(I)):
        G = oracle.cp_gradient_full(y, I, A, n)
        scale = np.linalg.norm(oracle.cp_gradient(y, I, A, n))
        assert np.linalg.norm(G) <= 1e-12 * scale


def test_gradient_step_descends():
    """eq. 2.15 along G (= -1/2 dD/da): D drops, to first order by 2 eta ||G||^2."""
    I, R = [6, 5, 7], 3
    p = cpsynth.make_problem(I, R, snr_db=10.0, seed=15, dtype=np.float64)
    A = [a.copy() for a in p.init]
    D0 = oracle.cp_cost(p.y, A)
    eta = 1e-6
    A1, G = oracle.cp_gradient_step(p.y, I, A, eta)
    D1 = oracle.cp_cost(p.y, A1)
    g2 = sum(float(np.sum(g * g)) for g in G)
    assert D1 < D0
    assert abs((D0 - D1) - 2 * eta * g2) <= 1e-3 * (2 * eta * g2)


def _nonneg_problem(I, R, seed, noise):
    rng = cpsynth.rng(seed, 7)
    A = [np.abs(rng.standard_normal((In, R))) + 0.1 for In in I]
    y = cpsynth.cp_model_vec(A)
    y = y + noise * np.abs(rng.standard_normal(y.shape)) * np.std(y)
    A0 = [np.abs(rng.standard_normal((In, R))) + 0.1 for In in I]
    return y, A, A0


def test_ntf_exact_factorisation_is_fixed_point():
    """At an exact nonnegative factorisation Y_(n) KR = A^(n) Gamma^(n), so
    eq. 2.18 multiplies every entry by one."""
    I, R = [5, 4, 6], 2
    y, A, _ = _nonneg_problem(I, R, 16, 0.0)
    tr = oracle.cp_ntf(y, I, A, iters=2)
    for n in range(len(I)):
        assert np.allclose(tr.A[n], A[n], rtol=1e-12, atol=1e-14)
    assert tr.fits[-1] > 1 - 1e-6


def test_ntf_monotone_nonnegative_and_fit_formula():
    """Multiplicative updates never raise D (Lee and Seung's auxiliary-function
    argument applies mode by mode) and keep the factors nonnegative; the cheap
    fit equals the explicit one."""
    I, R = [7, 6, 5, 4], 3
    y, _, A0 = _nonneg_problem(I, R, 17, 0.3)
    A = [a.copy() for a in A0]
    D = oracle.cp_cost(y, A)
    for _ in range(6):
        tr = oracle.cp_ntf(y, I, A, iters=1)
        A = tr.A
        Dn = oracle.cp_cost(y, A)
        assert Dn <= D * (1 + 1e-12)
        assert all(np.all(a >= 0) for a in A)
        assert abs(tr.fits[-1] - oracle.cp_fit_direct(y, A, np.ones(R))) <= 1e-9
        D = Dn


def test_sweep_backward_error_check():
    """The ALS parity check (tests/als_checks.py): zero for the oracle's own
    sweep, the size of the error for a planted one, and independent of the
    column scales that normalisation removes."""
    from als_checks import sweep_backward_errors
    I, R = [7, 6, 5, 4], 3
    p = cpsynth.make_problem(I, R, snr_db=20.0, seed=17, dtype=np.float64)
    tr = oracle.cp_als(p.y, I, p.init, iters=1)
    errs = sweep_backward_errors(p.y, I, p.init, tr.A)
    assert set(errs) == set(range(len(I)))
    assert max(errs.values()) <= 1e-12, errs
    scaled = [a * np.array([2.0, 0.5, 3.0])[None, :] for a in tr.A]
    assert max(sweep_backward_errors(p.y, I, p.init, scaled).values()) <= 1e-12
    for n in range(len(I)):
        bad = [a.copy() for a in tr.A]
        bad[n][0, 0] += 1e-3 * np.linalg.norm(bad[n])
        e = sweep_backward_errors(p.y, I, p.init, bad)
        assert e[n] > 1e-5, (n, e)
