"""Oracle O2: the Cauchy-matrix formula of Theorem 3.1, evaluated directly in FP64.

Test infrastructure only; the product path never imports it.

For L = L~ + rho v v^T (Def. 2.3) with L~ = U diag(lambda) U^T:
  z = U^T v                                   (Theorem 3.1)
  mu_i = roots of 1 + rho sum_j z_j^2 / (lambda_j - mu) = 0
                                              (Remark on the setup stage; Golub 1973)
  lambda and mu interlace                     (Lemma 4.1)
  x_i = -a_i U (mu_i I - Lambda)^{-1} z       (Lemma 4.2)
  X^T = -diag(a) C(mu, lambda) diag(z) U^T    (Theorem 3.1, eq. fwd_map)
so the coefficient of signal x on eigenvector i is
  y_i = -a_i sum_j z_j s_j / (mu_i - lambda_j),  s = U^T x  (Algorithm 1 steps 1, 2, 8).

Readings where the paper is silent:
* a_i normalises column i; its sign is chosen so that <u_pi(i), x_i> > 0, where
  pi pairs the i-th non-deflated root with the i-th non-deflated pole in
  ascending order (mu_i sits just above lambda_pi(i) for rho > 0, just below
  for rho < 0). This gives sign(a_i) = -sign(rho) sign(z_pi(i)).
* Deflated indices j (z_j ~ 0, Sec. 4) keep eigenpair (lambda_j, u_j); their
  coefficient is s_j.
* Output rows are in ascending eigenvalue order, a deflated row first on a tie.
* rho < 0 mirrors Lemma 4.1: mu_0 < lambda_0 and mu_i lies in (lambda_{i-1}, lambda_i).

Every root is bracketed by Lemma 4.1 and found by plain bisection on the
increasing function g(mu) = 1/rho + sum_j z_j^2 / (lambda_j - mu). A root is
held as (origin pole p, offset tau) with mu = lambda_p + tau and p the nearer
end of its bracket, and gaps are formed as
  mu - lambda_j = tau - (lambda_j - lambda_p),
with lambda_j - lambda_p from the product form in ``common.pole_differences``,
so no gap loses digits to cancellation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .common import deflation_mask, dct2, dct2_basis, path_eigenvalues, pole_differences


@dataclass
class CauchyPlan:
    n: int
    rho: float
    v: np.ndarray
    lam: np.ndarray          # (n,) path-graph eigenvalues
    z: np.ndarray            # (n,) z = U^T v
    deflated: np.ndarray     # (n,) bool
    poles: np.ndarray        # (K,) non-deflated pole indices, ascending
    origin: np.ndarray       # (K,) origin pole index of each root
    tau: np.ndarray          # (K,) mu_i - lambda_origin
    sign: np.ndarray         # (K,) sign of a_i
    a: np.ndarray            # (K,) normalisation with sign
    row_kind: np.ndarray     # (n,) 1 = root row, 0 = deflated row
    row_index: np.ndarray    # (n,) root number i, or deflated pole j
    eigenvalues: np.ndarray  # (n,) ascending eigenvalues of L

    @property
    def mu(self) -> np.ndarray:
        return self.lam[self.origin] + self.tau


def _secular_g(n, rho, z_nd, poles, origin, tau, d=None):
    """g(mu) = 1/rho + sum_j z_j^2/(lambda_j - mu) for mu = lambda_origin + tau (vectorised).

    ``d`` may pass the precomputed lambda_j - lambda_origin matrix.
    """
    if d is None:
        d = pole_differences(n, poles[None, :], origin[:, None])  # lambda_j - lambda_origin
    return 1.0 / rho + np.sum(z_nd[None, :] ** 2 / (d - tau[:, None]), axis=1)


def _bisect(n, rho, z_nd, poles, origin, lo, hi, max_iter=4000):
    """Bisection on tau in (lo, hi) with g(lo) < 0 <= g(hi); stops when no midpoint is left."""
    lo = lo.copy()
    hi = hi.copy()
    d_all = pole_differences(n, poles[None, :], origin[:, None])  # fixed over the iteration
    active = np.ones(lo.shape, dtype=bool)
    for _ in range(max_iter):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        mid = lo[idx] + 0.5 * (hi[idx] - lo[idx])
        done = (mid <= lo[idx]) | (mid >= hi[idx])
        active[idx[done]] = False
        idx, mid = idx[~done], mid[~done]
        if idx.size == 0:
            break
        g = _secular_g(n, rho, z_nd, poles, origin[idx], mid, d=d_all[idx])
        up = g >= 0.0
        hi[idx[up]] = mid[up]
        lo[idx[~up]] = mid[~up]
    else:
        raise RuntimeError("secular bisection did not converge")
    # return the end of the final bracket with the smaller |g| (lo may sit on a pole)
    with np.errstate(divide="ignore", invalid="ignore"):
        glo = np.abs(_secular_g(n, rho, z_nd, poles, origin, lo, d=d_all))
        ghi = np.abs(_secular_g(n, rho, z_nd, poles, origin, hi, d=d_all))
    glo = np.where(np.isfinite(glo), glo, np.inf)
    return np.where(ghi <= glo, hi, lo)


def make_plan(n: int, v, rho: float, roots=None, chunk: int = 256) -> CauchyPlan:
    """Setup stage (Remark in Sec. 3): lambda, z, deflation, mu and a.

    ``roots`` restricts the secular solve and normalisation to a subset of root
    numbers (for sampled checks at large n); the other entries stay NaN.
    """
    v = np.asarray(v, dtype=np.float64)
    if v.shape != (n,):
        raise ValueError("v must have length n")
    lam = path_eigenvalues(n)
    z = dct2(v[None, :])[0]
    deflated = deflation_mask(z, rho)
    poles = np.nonzero(~deflated)[0]
    K = poles.size
    z_nd = z[poles]
    znorm2 = float(np.sum(z_nd ** 2))

    origin = np.zeros(K, dtype=np.int64)
    tau = np.full(K, np.nan)
    sel = np.arange(K) if roots is None else np.asarray(sorted(set(int(r) for r in roots)), dtype=np.int64)
    for c0 in range(0, sel.size, chunk):
        ids = sel[c0:c0 + chunk]
        # Lemma 4.1 brackets, as (left pole, right pole or None)
        left = np.empty(ids.size, dtype=np.int64)
        right = np.empty(ids.size, dtype=np.int64)
        outer = np.zeros(ids.size, dtype=bool)
        for t, i in enumerate(ids):
            if rho > 0:
                left[t] = poles[i]
                if i + 1 < K:
                    right[t] = poles[i + 1]
                else:
                    right[t] = -1
                    outer[t] = True
            else:
                right[t] = poles[i]
                if i >= 1:
                    left[t] = poles[i - 1]
                else:
                    left[t] = -1
                    outer[t] = True
        org = np.empty(ids.size, dtype=np.int64)
        lo = np.empty(ids.size)
        hi = np.empty(ids.size)
        inner = ~outer
        if inner.any():
            # decide which half holds the root: g at the midpoint of the bracket
            gap = pole_differences(n, right[inner], left[inner])
            gmid = _secular_g(n, rho, z_nd, poles, left[inner], 0.5 * gap)
            in_left = gmid >= 0.0
            o = np.where(in_left, left[inner], right[inner])
            org[inner] = o
            lo[inner] = np.where(in_left, 0.0, -0.5 * gap)
            hi[inner] = np.where(in_left, 0.5 * gap, 0.0)
        if outer.any():
            if rho > 0:
                org[outer] = left[outer]
                lo[outer] = 0.0
                hi[outer] = rho * znorm2
            else:
                org[outer] = right[outer]
                lo[outer] = rho * znorm2
                hi[outer] = 0.0
        tau[ids] = _bisect(n, rho, z_nd, poles, org, lo, hi)
        origin[ids] = org

    # normalisation a_i = sign_i / sqrt(sum_j z_j^2 / (mu_i - lambda_j)^2)   (Theorem 3.1)
    sign = -np.sign(rho) * np.sign(z_nd) if K else np.zeros(0)
    a = np.full(K, np.nan)
    for c0 in range(0, sel.size, chunk):
        ids = sel[c0:c0 + chunk]
        gaps = tau[ids][:, None] - pole_differences(n, poles[None, :], origin[ids][:, None])
        a[ids] = sign[ids] / np.sqrt(np.sum(z_nd[None, :] ** 2 / gaps ** 2, axis=1))

    # merge root rows and deflated rows in ascending eigenvalue order
    mu = lam[origin] + tau if K else np.zeros(0)
    if roots is not None:
        # unsolved roots: place them at their pairing pole for ordering purposes
        mu = np.where(np.isnan(mu), lam[poles] if K else mu, mu)
    dpoles = np.nonzero(deflated)[0]
    values = np.concatenate([lam[dpoles], mu])
    kind = np.concatenate([np.zeros(dpoles.size, np.int64), np.ones(K, np.int64)])
    index = np.concatenate([dpoles, np.arange(K)])
    order = np.lexsort((kind, values))
    return CauchyPlan(n=n, rho=float(rho), v=v, lam=lam, z=z, deflated=deflated, poles=poles,
                      origin=origin, tau=tau, sign=sign, a=a, row_kind=kind[order],
                      row_index=index[order], eigenvalues=values[order])


def cauchy_rows(plan: CauchyPlan, rows) -> np.ndarray:
    """Rows of W = X^T U (so y = W s): W_ik = -a_i z_k / (mu_i - lambda_k); e_j for deflated rows."""
    n = plan.n
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((rows.size, n))
    for t, r in enumerate(rows):
        if plan.row_kind[r] == 0:
            out[t, plan.row_index[r]] = 1.0
        else:
            i = plan.row_index[r]
            gaps = plan.tau[i] - pole_differences(n, plan.poles, plan.origin[i])
            out[t, plan.poles] = -plan.a[i] * plan.z[plan.poles] / gaps
    return out


def transform(plan: CauchyPlan, x, rows=None, block: int = 1024) -> np.ndarray:
    """y = X^T x for each row of x (Algorithm 1: DCT-II, scale by z, Cauchy, scale by a).

    ``rows`` selects output coefficients (default: all n).
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    s = dct2(x)
    rows = np.arange(plan.n) if rows is None else np.asarray(rows, dtype=np.int64)
    y = np.empty((x.shape[0], rows.size))
    for r0 in range(0, rows.size, block):
        rr = rows[r0:r0 + block]
        y[:, r0:r0 + rr.size] = s @ cauchy_rows(plan, rr).T
    return y


def transform_matrix(plan: CauchyPlan) -> np.ndarray:
    """The full n x n matrix T = X^T (rows in ascending eigenvalue order): y = T x."""
    return cauchy_rows(plan, np.arange(plan.n)) @ dct2_basis(plan.n).T


def pruned_transform(plan: CauchyPlan, x, m_out: int, c_p: int) -> np.ndarray:
    """Pruned coefficients of Theorem 3.4: the first m_out entries of C^ s.

    W = -diag(a) C(mu, lambda) diag(z) maps the DCT coefficients s = U^T x to
    y = W s (Theorem 3.1). C^ keeps the upper-left c_p x c_p block of W and is
    zero elsewhere, so output i < m_out <= c_p is sum_{j < c_p} W_ij s_j. With
    c_p = n this is exactly the first m_out coefficients of the transform.
    """
    n = plan.n
    if not (1 <= m_out <= c_p <= n):
        raise ValueError("need 1 <= m_out <= c_p <= n")
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    s = dct2(x)
    w = cauchy_rows(plan, np.arange(m_out))
    return s[:, :c_p] @ w[:, :c_p].T


def pruning_bound(plan: CauchyPlan, x, c_p: int) -> np.ndarray:
    """Right-hand side of Theorem 3.4 per signal: ||s_{c_p+1:n}|| + ||W_hl s_{1:c_p}||, with
    W_hl the lower-left (n - c_p) x c_p block of W (the bound covers all n outputs, the
    pruned ones being zero beyond c_p)."""
    n = plan.n
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    s = dct2(x)
    w_hl = cauchy_rows(plan, np.arange(c_p, n))[:, :c_p]
    return np.linalg.norm(s[:, c_p:], axis=1) + np.linalg.norm(s[:, :c_p] @ w_hl.T, axis=1)
