"""The paper's own evaluation of the Cauchy product (Algorithm 1 steps 3-7, Sec. 4), FP64.

Test infrastructure only; the product path never imports it.

With s = z * DCT-II(x) (Algorithm 1 steps 1-2), the product p = C(mu, lambda) s is split
(pre-processing) into the column of the zero pole lambda_0 = 0, which stays explicit as
s_0 / mu_i, and the Cauchy product against the other poles. For a root in (0, 4), write
mu = 2 - 2 cos(theta). The poles lambda_j = 2 - 2 cos(pi j / n), j = 1..n-1, are the zeros of
the Chebyshev polynomial U_{n-1} in the variable 1 - lambda / 2. By Gastinel's proposition,
the rational function sum_j s_j / (x - cos(pi j / n)) equals h(x) / g(x) with
g = d_n U_{n-1} and h of degree n - 2. Interpolating h in the U basis (Lemma 4.3, a DST-I)
and substituting x = cos(theta) reduces the product to the trigonometric polynomial
(eq. trigo):

    sum_{j=1}^{n-1} s_j / (cos(theta) - cos(pi j / n))
        = sum_{l=1}^{n-1} c_l sin(l theta) / sin(n theta),
    c_l = 2 sum_{j=1}^{n-1} (-1)^(j+1) s_j sin(pi l j / n) / sin(pi j / n).

Here d_n = 2^-(n-1) has been cancelled between h and g, so it is never formed (it underflows
beyond n of about 1024). The paper evaluates the sine series with an NFST. Here it is summed
directly, which is the same quantity without the fast algorithm. Since mu - lambda_j
= 2 (cos(pi j / n) - cos(theta)),

    p_i = s_0 / mu_i - 1/2 * sum_l c_l sin(l theta_i) / sin(n theta_i),

and y_i = -a_i p_i (eq. fwd_map). Roots outside (0, 4) have no real angle: for rho > 0 the
largest, for rho < 0 the smallest (the paper isolates mu_n for rho > 0). Their rows are plain
sums, and deflated rows are the DCT coefficient itself, as in the other oracles.

Conditioning: when a root lies very close to a pole, sin(n theta) and the sine series both
nearly vanish. Their quotient then loses relative accuracy of order eps / |sin(n theta)|;
this is what makes the route ill-conditioned.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import cauchy
from .common import dct2, path_eigenvalues, pole_differences


def dst1_coefficients(s_rest: np.ndarray) -> np.ndarray:
    """c_l, l = 1..n-1, from s_j, j = 1..n-1 (rows), by the DST-I of Lemma 4.3 (after d_n
    cancels): c_l = 2 sum_j (-1)^(j+1) s_j sin(pi l j / n) / sin(pi j / n)."""
    s_rest = np.atleast_2d(s_rest)
    m = s_rest.shape[1]          # n - 1
    n = m + 1
    j = np.arange(1, n)
    h = ((-1.0) ** (j + 1)) * s_rest / np.sin(np.pi * j / n)
    # scipy's DST-I: y_k = 2 sum_{j=0}^{m-1} x_j sin(pi (j+1)(k+1) / (m+1))
    return scipy.fft.dst(h, type=1, axis=1)


def sine_series(c: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """sum_{l=1}^{n-1} c_l sin(l theta) for every row of c and every angle (direct NDST)."""
    c = np.atleast_2d(c)
    l = np.arange(1, c.shape[1] + 1)
    return c @ np.sin(np.outer(l, theta))


def transform(plan: cauchy.CauchyPlan, x) -> np.ndarray:
    """y = X^T x by Algorithm 1 with the trigonometric evaluation of the Cauchy product."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    n = plan.n
    sd = dct2(x)
    znd = np.where(plan.deflated, 0.0, plan.z)
    s = sd * znd[None, :]                                   # Algorithm 1 step 2
    lam = path_eigenvalues(n)
    c = dst1_coefficients(s[:, 1:])                        # steps 4-5
    y = np.empty((x.shape[0], n))
    for r in range(n):
        if plan.row_kind[r] == 0:                          # deflated: u_j itself
            y[:, r] = sd[:, plan.row_index[r]]
            continue
        i = plan.row_index[r]
        mu = plan.mu[i]
        a = plan.a[i]
        if 0.0 < mu < 4.0:
            theta = 2.0 * np.arctan2(np.sqrt(mu), np.sqrt(4.0 - mu))
            f = sine_series(c, np.array([theta]))[:, 0] / np.sin(n * theta)  # step 6
            p = s[:, 0] / mu - 0.5 * f                     # step 7 (compensation)
        else:                                              # the isolated root: a plain sum
            gaps = plan.tau[i] - pole_differences(n, np.arange(n), plan.origin[i])
            p = s @ (1.0 / gaps)
        y[:, r] = -a * p
    del lam
    return y
