"""Plain FP64 CPU oracle for the CP gradient (Section 2.2, Algorithm 1) and
CP_ALS (eq. 2.14, Section 4).  TEST INFRASTRUCTURE ONLY -- see the package
docstring for who may import it.

Everything here forms the explicit objects the fast method avoids: the
mode-n unfolding Y_(n) (Definition 2.2, Remark 2.1.2) and the explicit
Khatri-Rao matrix (Notation 2.1), multiplied with one matrix product.  There
is no blocking, fusion, split point or recursion of Algorithm 2 in here; the
fast method reaches the same numbers only up to rounding order, because
eqs. 3.7-3.10 and 3.19-3.22 are re-associations of the same sums.

Indices are 0-based in code; the paper is 1-based.  A tensor is passed as
vec(Y) (mode 1 fastest, eq. 2.1) plus its shape I; factors are (I_n, R)
float64 arrays.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np


def as_tensor(y: np.ndarray, I: Sequence[int]) -> np.ndarray:
    """N-D view Y[i_1, ..., i_N] of vec(Y) (eq. 2.1, column-major)."""
    return np.asarray(y, dtype=np.float64).reshape([int(v) for v in I], order="F")


def unfold(Y: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization Y_(n) (Definition 2.2 with r = [n] and
    c = [1..n-1, n+1..N] in increasing order, Remark 2.1.2): entry
    (i_n, j) with j = ivec of the remaining indices, column-major.
    Formed explicitly, as step 1-2 of Algorithm 1 does (permute + reshape)."""
    Yp = np.moveaxis(Y, n, 0)                         # permute(Y, [n, 1..n-1, n+1..N])
    return np.reshape(Yp, (Y.shape[n], -1), order="F")  # reshape to I_n x J_{-n}


def khatri_rao(mats: Sequence[np.ndarray]) -> np.ndarray:
    """Khatri-Rao product mats[0] (.) mats[1] (.) ... (Notation 2.1): column r
    is the Kronecker product of the r-th columns, so the LAST matrix's row
    index runs fastest.  Called with A^(N), ..., A^(1) (reverse mode order) its
    row index is the column-major ivec over the modes, matching Y_(n)."""
    R = mats[0].shape[1]
    rows = int(np.prod([m.shape[0] for m in mats]))
    out = np.empty((rows, R))
    for r in range(R):
        col = np.ones(1)
        for m in mats:
            col = np.kron(col, m[:, r])
        out[:, r] = col
    return out


def cp_gradient(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^(n) = Y_(n) (A^(N) (.) ... A^(n+1) (.) A^(n-1) ... (.) A^(1))
    (eq. 2.13 product term, Algorithm 1): explicit unfolding times explicit
    Khatri-Rao matrix, one fp64 matrix product."""
    Y = as_tensor(y, I)
    N = len(I)
    W = khatri_rao([A[m] for m in reversed(range(N)) if m != n])
    return unfold(Y, n) @ W


def cp_gradient_all(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray]) -> list[np.ndarray]:
    """All N gradients, each by Algorithm 1 (no sharing between modes)."""
    return [cp_gradient(y, I, A, n) for n in range(len(I))]


def cp_gradient_entry(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray], n: int,
                      i: int, r: int) -> float:
    """One entry g_r^(n)[i] of eq. 3.2: the slice of Y at i_n = i contracted
    with the Kronecker product of the r-th columns of the other factors.
    Used to check single sampled outputs on tensors too large for the full
    unfold-and-multiply."""
    Y = as_tensor(y, I)
    N = len(I)
    S = Y[(slice(None),) * n + (i,)]                # (N-1)-D slice at i_n = i (a view)
    t = np.ones(1)
    for m in reversed(range(N)):
        if m != n:
            t = np.kron(t, A[m][:, r])
    return float(np.reshape(S, -1, order="F") @ t)


def cp_gradient_entries(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray], n: int,
                        entries: Sequence[tuple[int, int]]) -> list[float]:
    """Entries g_r^(n)[i] of eq. 3.2 for the (i, r) pairs given, as
    cp_gradient_entry computes each one, but with each slice of Y at i_n = i
    formed (in FP64) only once and without an FP64 copy of the whole tensor,
    for tensors of several GB."""
    I = [int(v) for v in I]
    N = len(I)
    Y = np.asarray(y).reshape(I, order="F")            # view, no copy
    out, slices = [], {}
    for i, r in entries:
        if i not in slices:
            slices.clear()
            S = Y[(slice(None),) * n + (i,)]            # (N-1)-D slice at i_n = i (a view)
            slices[i] = np.reshape(S, -1, order="F").astype(np.float64)
        t = np.ones(1)
        for m in reversed(range(N)):
            if m != n:
                t = np.kron(t, np.asarray(A[m], dtype=np.float64)[:, r])
        out.append(float(slices[i] @ t))
    return out


def split_point(I: Sequence[int]) -> int:
    """n* = max{n : J_n <= K_n} of Algorithm 2 (step 1), J_n = I_1..I_n and
    K_n = I_{n+1}..I_N, 1-based, with "<=" as printed.  When no n satisfies
    it (I_1 > I_2..I_N) or it would be N, the value is clamped into
    [1, N-1] so that both sides of the split are non-empty."""
    N = len(I)
    best = 0
    for n in range(1, N + 1):
        J = int(np.prod(I[:n]))
        K = int(np.prod(I[n:])) if n < N else 1
        if J <= K:
            best = n
    return min(max(best, 1), N - 1)


def als_mode_order(I: Sequence[int], k: int | None = None) -> list[int]:
    """Update order of the fast ALS (Section 4), 0-based: with k = n*,
    modes k-1, k-2, ..., 0 and then k, k+1, ..., N-1 (paper: n*, n*-1, ..., 1,
    n*+1, ..., N)."""
    N = len(I)
    if k is None:
        k = split_point(I)
    return list(range(k - 1, -1, -1)) + list(range(k, N))


def gram_hadamard(A: Sequence[np.ndarray], skip: int | None) -> np.ndarray:
    """Hadamard product over m != skip of A^(m)T A^(m) (eq. 2.13/2.14)."""
    R = A[0].shape[1]
    V = np.ones((R, R))
    for m, Am in enumerate(A):
        if m != skip:
            V = V * (Am.T @ Am)
    return V


def cp_full(A: Sequence[np.ndarray], lam: np.ndarray | None = None) -> np.ndarray:
    """vec of the CP model sum_r lam_r a_r^(1) o ... o a_r^(N) (eq. 2.7),
    formed as A^(1) (A^(N) (.) ... (.) A^(2))^T per Definition 2.4."""
    R = A[0].shape[1]
    lam = np.ones(R) if lam is None else np.asarray(lam, dtype=np.float64)
    N = len(A)
    if N == 1:
        return A[0] @ lam
    W = khatri_rao([A[m] for m in reversed(range(1, N))])
    Y1 = (A[0] * lam[None, :]) @ W.T                # mode-1 unfolding of the model
    return np.reshape(Y1, -1, order="F")


def cp_fit_direct(y: np.ndarray, A: Sequence[np.ndarray], lam: np.ndarray) -> float:
    """fit = 1 - ||Y - Yhat||_F / ||Y||_F with Yhat formed explicitly."""
    y = np.asarray(y, dtype=np.float64)
    return 1.0 - float(np.linalg.norm(y - cp_full(A, lam)) / np.linalg.norm(y))


def _solve_normal(G: np.ndarray, V: np.ndarray) -> np.ndarray:
    """A = G V^dagger (eq. 2.14).  V is symmetric PSD; Cholesky solve when V is
    positive definite, else the eigen pseudo-inverse with eigenvalues below
    R * eps * max|lambda| dropped."""
    try:
        L = np.linalg.cholesky(V)
        # A V = G  ->  V A^T = G^T  (V symmetric)
        Z = np.linalg.solve(L, G.T)
        return np.linalg.solve(L.T, Z).T
    except np.linalg.LinAlgError:
        w, Q = np.linalg.eigh(V)
        tol = V.shape[0] * np.finfo(np.float64).eps * max(np.max(np.abs(w)), 1e-300)
        winv = np.where(w > tol, 1.0 / np.where(w > tol, w, 1.0), 0.0)
        return G @ (Q * winv[None, :]) @ Q.T


@dataclasses.dataclass
class AlsTrace:
    A: list[np.ndarray]
    lam: np.ndarray
    fits: list[float]            # fit after each sweep (cheap formula)
    fits_direct: list[float]     # fit after each sweep (explicit Yhat), if requested


def cp_als(y: np.ndarray, I: Sequence[int], A0: Sequence[np.ndarray], iters: int,
           order: Sequence[int] | None = None, direct_fit: bool = False) -> AlsTrace:
    """Plain CP_ALS (eq. 2.14) with the fast ALS update order of Section 4.

    Each sweep visits the modes in ``order`` (default: als_mode_order(I)).
    For mode n: G = Y_(n) KR (Algorithm 1, explicit), V = Hadamard of the
    other modes' Grams, A^(n) = G V^dagger, then the columns are normalised:
    lam_r = ||a_r^(n)||_2 and a_r^(n) /= lam_r (a zero column is left as is
    with lam_r = 0).  The model is sum_r lam_r a_r^(1) o ... o a_r^(N).

    The fit after a sweep uses the last mode's gradient, as the fast ALS has
    it at hand: <Y, Yhat> = sum_r lam_r a_r^(last)T g_r^(last) and
    ||Yhat||^2 = lam^T (Hadamard of all Grams) lam, so
    fit = 1 - sqrt(max(0, ||Y||^2 - 2<Y,Yhat> + ||Yhat||^2)) / ||Y||.
    """
    N = len(I)
    A = [np.array(a, dtype=np.float64, copy=True) for a in A0]
    R = A[0].shape[1]
    lam = np.ones(R)
    if order is None:
        order = als_mode_order(I)
    yv = np.asarray(y, dtype=np.float64)
    normY2 = float(yv @ yv)
    fits, fitsd = [], []
    for _ in range(iters):
        G = None
        for n in order:
            G = cp_gradient(yv, I, A, n)
            V = gram_hadamard(A, skip=n)
            An = _solve_normal(G, V)
            nrm = np.linalg.norm(An, axis=0)
            lam = nrm.copy()
            safe = np.where(nrm > 0, nrm, 1.0)
            A[n] = An / safe[None, :]
        last = order[-1]
        inner = float(np.sum(lam * np.sum(A[last] * G, axis=0)))
        model2 = float(lam @ gram_hadamard(A, skip=None) @ lam)
        res2 = max(0.0, normY2 - 2.0 * inner + model2)
        fits.append(1.0 - np.sqrt(res2) / np.sqrt(normY2))
        if direct_fit:
            fitsd.append(cp_fit_direct(yv, A, lam))
    return AlsTrace(A=A, lam=lam, fits=fits, fits_direct=fitsd)


# ---- consumers of the gradient (Section 2.2) --------------------------------------
def cp_cost(y: np.ndarray, A: Sequence[np.ndarray]) -> float:
    """D = ||Y - Yhat||_F^2 (eq. 2.12), Yhat the CP model of the factors (no lambda)."""
    y = np.asarray(y, dtype=np.float64)
    r = y - cp_full(A)
    return float(r @ r)


def cp_gradient_full(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^(n) of eq. 2.13 with the model term: E_(n) KR = Y_(n) KR - A^(n) Gamma^(n),
    Gamma^(n) = Hadamard_{k != n} A^(k)T A^(k).  dD/dA^(n) = -2 G^(n)."""
    return cp_gradient(y, I, A, n) - np.asarray(A[n], dtype=np.float64) @ gram_hadamard(A, skip=n)


def cp_gradient_step(y: np.ndarray, I: Sequence[int], A: Sequence[np.ndarray], eta: float):
    """One all-at-once first-order step (eq. 2.15): every gradient of eq. 2.13 at
    the current factors, then a <- a + eta G for all modes at once (G is -1/2 the
    derivative of D, so this is a <- a - (eta/2) dD/da).  Returns (new factors,
    gradients)."""
    A = [np.asarray(a, dtype=np.float64) for a in A]
    G = [cp_gradient_full(y, I, A, n) for n in range(len(I))]
    return [A[n] + eta * G[n] for n in range(len(I))], G


@dataclasses.dataclass
class NtfTrace:
    A: list[np.ndarray]
    fits: list[float]            # fit after each sweep (cheap formula)


def cp_ntf(y: np.ndarray, I: Sequence[int], A0: Sequence[np.ndarray], iters: int,
           order: Sequence[int] | None = None) -> NtfTrace:
    """Multiplicative nonnegative CP updates (eq. 2.18) in the fast ALS mode
    order of Section 4 (each mode uses the factors updated before it):
        A^(n) <- A^(n) * (Y_(n) KR) / (A^(n) Gamma^(n)),
    elementwise; an entry whose denominator is not positive is left as is.
    No normalisation (the model is sum_r a_r^(1) o ... o a_r^(N)).  The fit after
    a sweep uses the last mode's gradient as in cp_als, with lambda = 1."""
    N = len(I)
    A = [np.array(a, dtype=np.float64, copy=True) for a in A0]
    if order is None:
        order = als_mode_order(I)
    yv = np.asarray(y, dtype=np.float64)
    normY2 = float(yv @ yv)
    fits = []
    for _ in range(iters):
        G = None
        for n in order:
            G = cp_gradient(yv, I, A, n)
            D = A[n] @ gram_hadamard(A, skip=n)
            A[n] = np.where(D > 0, A[n] * G / np.where(D > 0, D, 1.0), A[n])
        last = order[-1]
        inner = float(np.sum(A[last] * G))
        model2 = float(np.sum(gram_hadamard(A, skip=None)))
        fits.append(1.0 - np.sqrt(max(0.0, normY2 - 2.0 * inner + model2)) / np.sqrt(normY2))
    return NtfTrace(A=A, fits=fits)
