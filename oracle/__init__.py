"""FP64 CPU oracle for the CP gradient and CP_ALS.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls anything here, and this
package imports nothing from the product.

Pins (all in ``tests/test_oracle.py``; none re-types the oracle's own code):
  * brute force of the elementwise sum (eq. 3.2) on tiny tensors;
  * the closed form for an exact CP tensor (eq. 2.13 with E = 0);
  * the invariant tr(A^(n)T G^(n)) = sum_r Y x {a_r} for every n (eq. 2.6);
  * N = 2 reduces to the matrix products Y A2 and Y^T A1;
  * a hand-computed integer worked example (tests/golden/);
  * ALS: Eckart-Young on matrices (N = 2), fit -> 1 on noiseless low-rank
    tensors, monotone cost, the cheap fit formula against the explicit one;
  * the cost gradient of eq. 2.13 against central finite differences of
    D (eq. 2.12), zero at an exact CP factorisation; a small first-order step
    (eq. 2.15) lowers D;
  * multiplicative NTF (eq. 2.18): an exact nonnegative factorisation is a
    fixed point, D never rises, factors stay nonnegative.
"""
from .cp_oracle import (  # noqa: F401
    unfold, khatri_rao, cp_gradient, cp_gradient_all, cp_gradient_entry, cp_gradient_entries,
    split_point, als_mode_order, gram_hadamard, cp_full, cp_fit_direct,
    cp_als, AlsTrace, cp_cost, cp_gradient_full, cp_gradient_step, cp_ntf, NtfTrace,
)
