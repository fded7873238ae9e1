"""The leaf-level Chebyshev far field of the hierarchical Cauchy mode, checked in FP64 on the host.

The hierarchical mode evaluates W = X^T U (Theorem 3.1, W_rj = -a_r z_j / (mu_r - lambda_j)) as
an exact near field (target leaf I against source leaves I-1..I+1) plus a far field
Q K P: P holds the sources' z-weighted Lagrange weights at the R = 12 Chebyshev nodes of their
leaf, K the kernel 1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph) sampled at the nodes of every
pair of leaves at least one leaf apart, Q the targets' -a-weighted Lagrange weights. This test
builds the three factors in FP64 from the interpolation definition (not from the CUDA code) and
compares Q K P with the far part of W from the oracle: the interpolation error for boxes one
box apart decays like (3 + sqrt 8)^-R, about 7e-10 at R = 12.
"""
import numpy as np
import pytest

from oracle import cauchy
from synthetic import random_unit_v, self_loop_v

LEAF, R = 64, 12


def cheb_nodes():
    return np.cos((2 * np.arange(R) + 1) * np.pi / (2 * R))


def lagrange(u):
    """L[k, a] = S_a(u_k), the Lagrange basis on the Chebyshev nodes of [-1, 1]."""
    t = cheb_nodes()
    u = np.atleast_1d(u)[:, None]
    out = np.ones((u.shape[0], R))
    for a in range(R):
        for b in range(R):
            if b != a:
                out[:, a] *= (u[:, 0] - t[b]) / (t[a] - t[b])
    return out


def far_field_factors(plan):
    n = plan.n
    nleaf = n // LEAF
    h = np.pi / nleaf
    th = np.pi * np.arange(n) / n
    src_leaf = np.arange(n) // LEAF
    zf = np.where(plan.deflated, 0.0, plan.z)
    # P: sources
    P = np.zeros((nleaf * R, n))
    u_src = (th - (src_leaf + 0.5) * h) / (0.5 * h)
    Ls = lagrange(u_src)
    for j in range(n):
        P[src_leaf[j] * R:(src_leaf[j] + 1) * R, j] = zf[j] * Ls[j]
    # K: leaf pairs at least one leaf apart
    nodes = ((np.arange(nleaf)[:, None] + 0.5) * h + 0.5 * h * cheb_nodes()[None, :]).ravel()
    ph, tj = nodes[:, None], nodes[None, :]
    with np.errstate(divide="ignore"):  # the diagonal (a leaf with itself) is masked below
        K = 1.0 / (4.0 * np.sin(0.5 * (ph + tj)) * np.sin(0.5 * (ph - tj)))
    leaf_of_node = np.repeat(np.arange(nleaf), R)
    K[np.abs(leaf_of_node[:, None] - leaf_of_node[None, :]) <= 1] = 0.0
    # Q: root rows with a real angle
    Q = np.zeros((n, nleaf * R))
    tgt_leaf = np.full(n, -1)
    mu = plan.mu
    for r in range(n):
        if plan.row_kind[r] == 0:
            continue
        i = plan.row_index[r]
        if not 0.0 < mu[i] < 4.0:
            continue
        phi = 2.0 * np.arcsin(np.sqrt(mu[i]) / 2.0)
        lf = min(max(int(np.floor(phi / h)), 0), nleaf - 1)
        tgt_leaf[r] = lf
        u = (phi - (lf + 0.5) * h) / (0.5 * h)
        Q[r, lf * R:(lf + 1) * R] = -plan.a[i] * lagrange(u)[0]
    return P, K, Q, src_leaf, tgt_leaf


@pytest.mark.parametrize("n", [256, 1024, 4096])
@pytest.mark.parametrize("kind", ["dense_v", "self_loop"])
def test_leaf_level_far_field_matches_the_far_part_of_w(n, kind):
    v, rho = (random_unit_v(n, seed=1), 2.0) if kind == "dense_v" else (self_loop_v(n, 0), -0.5)
    plan = cauchy.make_plan(n, v, rho)
    W = cauchy.cauchy_rows(plan, np.arange(n))
    P, K, Q, src_leaf, tgt_leaf = far_field_factors(plan)
    approx = Q @ (K @ P)
    far = (tgt_leaf[:, None] >= 0) & (np.abs(tgt_leaf[:, None] - src_leaf[None, :]) >= 2)
    exact = np.where(far, W, 0.0)
    rel = np.linalg.norm(approx - exact, axis=1) / np.linalg.norm(W, axis=1)
    assert rel.max() < 1e-8, rel.max()
    # the far field carries a measurable part of the rows, so the check is not vacuous
    if n >= 1024:
        frac = np.linalg.norm(exact, axis=1) / np.linalg.norm(W, axis=1)
        assert np.median(frac) > 1e-3


def test_interpolation_rate_with_the_degree():
    """The error of the sampled kernel between boxes one box apart falls like (3 + sqrt 8)^-R."""
    h = np.pi / 16
    c_i, c_j = 5.5 * h, 7.5 * h  # centres two boxes apart: one box between them
    u = np.linspace(-1, 1, 41)
    ph, th = c_i + 0.5 * h * u, c_j + 0.5 * h * u
    exact = 1.0 / (2 * np.cos(th)[None, :] - 2 * np.cos(ph)[:, None])
    errs = []
    for deg in (4, 8, 12):
        t = np.cos((2 * np.arange(deg) + 1) * np.pi / (2 * deg))
        def lag(x):
            out = np.ones((x.size, deg))
            for a in range(deg):
                for b in range(deg):
                    if b != a:
                        out[:, a] *= (x - t[b]) / (t[a] - t[b])
            return out
        Kn = 1.0 / (2 * np.cos(c_j + 0.5 * h * t)[None, :] - 2 * np.cos(c_i + 0.5 * h * t)[:, None])
        approx = lag(u) @ Kn @ lag(u).T
        errs.append(np.abs(approx - exact).max() / np.abs(exact).max())
    assert errs[2] < 1e-8
    assert errs[0] > errs[1] > errs[2]
