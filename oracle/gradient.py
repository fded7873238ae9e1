"""Gradients of the DCT+ transform in FP64 (the derivatives the backward pass returns).

Test infrastructure only; the product path never imports it.

For y_b = X^T x_b (Theorem 3.1) and an upstream gradient g_b = dLoss/dy_b:

* with respect to the signal: X is orthogonal, so dLoss/dx_b = X g_b, the
  inverse transform (the backward pass the paper obtains by inverting the
  forward steps, Sec. 3);
* with respect to rho and v: the eigenvectors of L = L~ + rho v v^T (Def. 2.3)
  move with the update. First-order perturbation of a symmetric eigenproblem
  with distinct eigenvalues gives dx_i = sum_{k != i} x_k (x_k^T dL x_i) /
  (mu_i - mu_k), with dL = v v^T drho + rho (dv v^T + v dv^T). Writing
  w = X^T v and K_ik = 1 / (mu_i - mu_k) for k != i (K_ii = 0):

      dLoss/drho = sum_b sum_i g_bi w_i sum_k K_ik w_k y_bk
      dLoss/dv   = rho X sum_b r_b,
      r_b = y_b * (K^T (g_b * w)) + g_b * (K (y_b * w))      (elementwise *).

  The eigenvalues themselves do not enter y, so their derivatives are not needed.
For roots of the secular equation w_i = -a_i / rho (Lemma 4.2 with the secular
equation); the code below forms w = X^T v directly.
"""
from __future__ import annotations

import numpy as np

from . import cauchy


def backward_x(plan: cauchy.CauchyPlan, g) -> np.ndarray:
    """dLoss/dx = X g for each row g of ``g`` (rows of X^T are the eigenvectors)."""
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    return g @ cauchy.transform_matrix(plan)


def cauchy_k(plan: cauchy.CauchyPlan) -> np.ndarray:
    """K_ik = 1 / (mu_i - mu_k) for i != k, 0 on the diagonal (rows in output order)."""
    mu = plan.eigenvalues
    d = mu[:, None] - mu[None, :]
    k = np.zeros_like(d)
    off = ~np.eye(plan.n, dtype=bool)
    k[off] = 1.0 / d[off]
    return k


def parameter_gradients(plan: cauchy.CauchyPlan, x, g):
    """(dLoss/drho, dLoss/dv) for signals x (rows) and upstream gradients g (rows)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    t = cauchy.transform_matrix(plan)          # X^T
    y = x @ t.T
    w = t @ plan.v                             # X^T v
    k = cauchy_k(plan)
    p = (y * w) @ k.T                          # row b: K (y_b * w)
    q = (g * w) @ k                            # row b: K^T (g_b * w)
    grad_rho = float(np.sum(g * w * p))
    r = y * q + g * p
    grad_v = plan.rho * (r.sum(axis=0) @ t)    # rho X sum_b r_b
    return grad_rho, grad_v
