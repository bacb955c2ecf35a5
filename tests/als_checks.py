"""Parity check of one computed CP_ALS sweep (eq. 2.14) against the oracle,
independent of the normal equations' conditioning.

A forward comparison of the factors amplifies the gradient's rounding by the
condition number of V = Hadamard_{m != n} A^(m)T A^(m): at ill-conditioned
iterates even the FP32 path's factors differ from the FP64 ones by more than
1e-5 after one sweep.  The backward error does not: for each mode n, in the
sweep's order, the oracle forms G^(n) = Y_(n) KR and V from the factors the
update of n saw (the modes updated earlier in the sweep at their new values,
the others at their starting values), and the check takes

    min_s || A^(n) diag(s) V - G^(n) ||_F / || G^(n) ||_F,

the relative residual of the computed (column-normalised) factor in the
oracle's normal equations, the column scales s free because the
normalisation removes them.  An exact solve of an exact gradient gives zero;
a gradient with relative error e gives about e."""
import numpy as np

import oracle


def sweep_backward_errors(y, I, A_start, A_end, order=None):
    """{mode: relative residual} for one sweep from A_start that produced A_end."""
    if order is None:
        order = oracle.als_mode_order(I)
    cur = [np.asarray(a, dtype=np.float64).copy() for a in A_start]
    R = cur[0].shape[1]
    out = {}
    for n in order:
        G = oracle.cp_gradient(y, I, cur, n)
        V = oracle.gram_hadamard(cur, skip=n)
        An = np.asarray(A_end[n], dtype=np.float64)
        M = np.stack([np.outer(An[:, r], V[r, :]).ravel() for r in range(R)], axis=1)
        s, *_ = np.linalg.lstsq(M, G.ravel(), rcond=None)
        out[n] = float(np.linalg.norm(M @ s - G.ravel()) / np.linalg.norm(G))
        cur[n] = An
    return out
