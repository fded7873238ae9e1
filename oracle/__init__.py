"""FP64 CPU oracle for the Fast DCT+ transform — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package. The product library
(``paper_2409_08970_gb300``) never imports it, and this package never imports
the product: the two share no code. Inputs come from ``synthetic``.

Two independent evaluations of the same transform y = X^T x:

* ``definition`` (O1): dense L~ + rho v v^T, cyclic Jacobi eigensolver in plain C,
  orientation rule, naive matrix-vector product (NMVP).
* ``cauchy`` (O2): the factorisation of Theorem 3.1 evaluated term by term —
  DCT-II by direct cosine sums, secular roots by bisection inside the
  Lemma 4.1 brackets, normalisation, and the Cauchy sum.
* ``gradient``: derivatives of the transform with respect to the signal, rho and
  v (inverse transform; first-order eigenvector perturbation).
* ``nfst_route``: the paper's own evaluation of the Cauchy product (pre-processing,
  DST-I, trigonometric series over sin(n theta)), with a direct sum in place of the NFST.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force at n <= 8, O1 against O2).
"""
from . import cauchy, common, definition, gradient, nfst_route  # noqa: F401
from ._native import build as build_native  # noqa: F401
