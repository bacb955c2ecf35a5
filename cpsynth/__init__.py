"""Seeded synthetic inputs shared by the oracle checks, the CUDA parity tests,
the smoke test and the benchmark.

This module only draws random numbers and assembles the CP model of
Definition 2.4 (eq. 2.7) as a data source; it computes no gradient, no
unfolding product and no ALS step, so the oracle and the CUDA path can both
consume its output without sharing any of the method's arithmetic.

Conventions (Section 2, eq. 2.1): a tensor of shape I = [I_1..I_N] is held as
its vectorisation vec(Y), a 1-D array in which mode 1 runs fastest
(column-major, MATLAB order).  A factor A^(n) is an I_n x R matrix; we hold it
as a numpy array of shape (I_n, R) and hand it to the device in column-major
order (ld = I_n), which is ``A.T`` made contiguous.

Workloads follow the random-tensor experiments of Section 5: random CP
models of order 3..7 with equal or mixed mode sizes, a rank R, and additive
Gaussian noise at a stated SNR.  The paper uses no public dataset.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

DEFAULT_SEED = 20120406


def rng(seed: int, *stream: int) -> np.random.Generator:
    """Independent PCG64 stream for (seed, stream...)."""
    ss = np.random.SeedSequence(entropy=int(seed), spawn_key=tuple(int(s) for s in stream))
    return np.random.default_rng(ss)


def gaussian_factors(I: Sequence[int], R: int, seed: int, stream: int = 0,
                     collinearity: float | None = None) -> list[np.ndarray]:
    """N(0,1) factors A^(n) of shape (I_n, R) in float64.

    With ``collinearity=c`` each row of A^(n) is drawn with covariance
    C = (1-c) I + c 11^T and the columns are then scaled to unit norm, so
    distinct columns have expected cosine c (the collinear-factor case the
    paper mentions at the end of Section 5).
    """
    out = []
    for n, In in enumerate(I):
        g = rng(seed, stream, n)
        Z = g.standard_normal((int(In), R))
        if collinearity is not None and R > 1:
            C = (1.0 - collinearity) * np.eye(R) + collinearity * np.ones((R, R))
            L = np.linalg.cholesky(C)
            Z = Z @ L.T
            Z = Z / np.linalg.norm(Z, axis=0, keepdims=True)
        out.append(Z)
    return out


def cp_model_vec(factors: Sequence[np.ndarray], out_dtype=np.float64,
                 weights: np.ndarray | None = None) -> np.ndarray:
    """vec of sum_r w_r a_r^(1) o ... o a_r^(N)  (eq. 2.7), built slab by slab
    over the last mode so that large tensors never need an fp64 copy."""
    N = len(factors)
    I = [f.shape[0] for f in factors]
    R = factors[0].shape[1]
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    total = int(np.prod(I))
    out = np.empty(total, dtype=out_dtype)
    if N == 1:
        out[:] = factors[0] @ w
        return out
    # head = columnwise outer product over modes 1..N-1, laid out column-major
    head = (factors[0] * w[None, :]).copy()          # (I_1, R)
    for n in range(1, N - 1):
        # row index of the new head is j_old + J_old * i_n (mode 1 fastest)
        head = np.einsum("ar,br->bar", head, factors[n]).reshape(-1, R)
    J = head.shape[0]
    last = factors[N - 1]
    step = max(1, (1 << 24) // max(J, 1))
    for i0 in range(0, I[N - 1], step):
        i1 = min(I[N - 1], i0 + step)
        slab = head @ last[i0:i1].T                  # (J, i1-i0), column i = slab for i_N=i
        out[i0 * J:i1 * J] = slab.T.reshape(-1)
    return out


def add_noise(y: np.ndarray, snr_db: float | None, seed: int, stream: int = 9) -> np.ndarray:
    """y + sigma * E with E ~ N(0,1) i.i.d. and sigma chosen so that
    ||y||^2 / (sigma^2 * numel) = 10^(snr/10) (expected noise power)."""
    if snr_db is None:
        return y
    sig2 = float(np.dot(y.astype(np.float64), y.astype(np.float64))) / (y.size * 10.0 ** (snr_db / 10.0))
    sigma = math.sqrt(sig2)
    g = rng(seed, stream)
    chunk = 1 << 24
    for s in range(0, y.size, chunk):
        e = g.standard_normal(min(chunk, y.size - s))
        y[s:s + e.size] += (sigma * e).astype(y.dtype)
    return y


@dataclasses.dataclass
class Problem:
    """One synthetic CP problem: tensor, true factors and an ALS start."""
    I: list[int]
    R: int
    y: np.ndarray                  # vec(Y), mode 1 fastest
    factors: list[np.ndarray]      # true factors (float64)
    init: list[np.ndarray]         # seeded N(0,1) start for ALS (float64)
    dtype: type


def make_problem(I: Sequence[int], R: int, *, snr_db: float | None = 20.0, seed: int = DEFAULT_SEED,
                 dtype=np.float32, collinearity: float | None = None) -> Problem:
    """Rank-R CP model with N(0,1) (or collinear) factors plus Gaussian noise.

    The tensor is rounded to ``dtype`` once; both the oracle and the device
    consume that rounded tensor (and the rounded factors), so parity compares
    the same inputs.
    """
    I = [int(v) for v in I]
    fac = gaussian_factors(I, R, seed, stream=1, collinearity=collinearity)
    y = cp_model_vec(fac, out_dtype=np.float64 if dtype == np.float64 else np.float32)
    y = add_noise(y, snr_db, seed)
    y = y.astype(dtype, copy=False)
    init = gaussian_factors(I, R, seed, stream=2)
    fac = [f.astype(dtype).astype(np.float64) for f in fac]
    init = [f.astype(dtype).astype(np.float64) for f in init]
    return Problem(I=I, R=R, y=y, factors=fac, init=init, dtype=dtype)


def random_tensor(I: Sequence[int], seed: int = DEFAULT_SEED, dtype=np.float32, stream: int = 5) -> np.ndarray:
    """Plain N(0,1) tensor (no low-rank structure), vec layout.  Drawn in
    chunks (the same values as one draw of the whole length), so that a large
    tensor never needs an FP64 copy."""
    g = rng(seed, stream)
    n = int(np.prod(I))
    out = np.empty(n, dtype=dtype)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        out[s:s + chunk] = g.standard_normal(min(chunk, n - s))
    return out


def random_factors(I: Sequence[int], R: int, seed: int = DEFAULT_SEED, dtype=np.float32,
                   stream: int = 6) -> list[np.ndarray]:
    """N(0,1) factors rounded to ``dtype`` and returned as float64 arrays."""
    return [f.astype(dtype).astype(np.float64) for f in gaussian_factors(I, R, seed, stream=stream)]


# Workload catalogue (Section 5 shapes, scaled to the GPU).  Each entry:
# name -> (I, R, snr_db, dtype, collinearity, als_iters)
WORKLOADS = {
    "cp3d_30x40x50_r5_fp64": ([30, 40, 50], 5, 20.0, np.float64, None, 10),
    "cp4d_100_r10_fp32": ([100, 100, 100, 100], 10, 20.0, np.float32, None, 50),
    "cp7d_15_r10_fp32": ([15] * 7, 10, 30.0, np.float32, 0.5, 30),
    "cp7d_15_r20_fp32": ([15] * 7, 20, 30.0, np.float32, 0.5, 30),
    "cp5d_60_r32_fp32": ([60] * 5, 32, 20.0, np.float32, None, 10),
    "cp5d_60_r64_fp32": ([60] * 5, 64, 20.0, np.float32, None, 10),
}


def workload(name: str, seed: int = DEFAULT_SEED) -> Problem:
    I, R, snr, dt, col, _ = WORKLOADS[name]
    return make_problem(I, R, snr_db=snr, seed=seed, dtype=dt, collinearity=col)


def batched_shapes(count: int = 256, seed: int = DEFAULT_SEED, orders=(3, 4, 5), size_range=(8, 64),
                   rank_range=(4, 32)) -> list[tuple[list[int], int]]:
    """Shapes and ranks of the batched workload: order N uniform in `orders`,
    every I_n uniform in `size_range` (inclusive), rank R uniform in
    `rank_range` (inclusive), one (I, R) per member."""
    g = rng(seed, 77)
    out = []
    for _ in range(count):
        N = int(g.choice(orders))
        I = [int(v) for v in g.integers(size_range[0], size_range[1] + 1, size=N)]
        R = int(g.integers(rank_range[0], rank_range[1] + 1))
        out.append((I, R))
    return out


def batched_workload(count: int = 256, seed: int = DEFAULT_SEED, orders=(3, 4, 5), size_range=(8, 64),
                     rank_range=(4, 32), snr_db: float = 20.0, dtype=np.float32) -> list[Problem]:
    """Many independent CP problems from one seed (shapes and ranks from
    batched_shapes), each a rank-R N(0,1) CP model plus Gaussian noise at
    `snr_db`, with its own seeded ALS start."""
    return [make_problem(I, R, snr_db=snr_db, seed=seed + 1 + b, dtype=dtype)
            for b, (I, R) in enumerate(batched_shapes(count, seed, orders, size_range, rank_range))]
