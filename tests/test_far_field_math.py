"""The Chebyshev far field of the hierarchical Cauchy mode, checked in FP64 on the host: the
leaf-level form (one dense leaf-to-leaf kernel matrix) and the multilevel tree the mode runs.

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


# ------------------------------------------------------------------ multilevel far field
#
# The hierarchical mode's far field is a 1-D fast multipole tree over the angle boxes:
# leaf moments (P2M, the factor P above) are re-expanded up the tree (M2M: the parent's
# Lagrange basis at its children's nodes, exact for polynomials of the degree), every box
# takes the kernel samples against the boxes of its interaction list (M2L: at least one box
# apart, parents adjacent; at the top level of 4 boxes, every box at least one apart), and
# the local expansions come down to the leaves (L2L, the transposed re-expansion), where the
# targets' weights Q read them. These factors are rebuilt here from that definition.

def child_reexpansion():
    """E[k][a, b] = S_a((x_b + 2k - 1) / 2): the parent's basis at child k's nodes (k = 0 left)."""
    t = cheb_nodes()
    return [lagrange((t + 2 * k - 1) / 2.0).T for k in (0, 1)]


def interaction_list(level_boxes, b, top):
    if top:
        return [c for c in range(level_boxes) if abs(c - b) >= 2]
    return [c for c in (b - 3, b - 2, b + 2, b + 3)
            if 0 <= c < level_boxes and abs(c // 2 - b // 2) <= 1]


def multilevel_far_operator(n):
    """Matrix F with leaf locals = F (leaf moments), both (nleaf R) long, built level by level."""
    nleaf = n // LEAF
    E = child_reexpansion()
    levels = []
    nb = nleaf
    while nb >= 4:
        levels.append(nb)
        nb //= 2
    # up: U[l] maps leaf moments to level-l moments
    U = [np.eye(nleaf * R)]
    for l in range(1, len(levels)):
        nb = levels[l]
        step = np.zeros((nb * R, levels[l - 1] * R))
        for p in range(nb):
            for k in (0, 1):
                step[p * R:(p + 1) * R, (2 * p + k) * R:(2 * p + k + 1) * R] = E[k]
        U.append(step @ U[-1])
    F = np.zeros((nleaf * R, nleaf * R))
    downs = [np.eye(nleaf * R)]  # downs[l] maps level-l locals to leaf locals (L2L chains)
    for l in range(1, len(levels)):
        nb_child, nb = levels[l - 1], levels[l]
        step = np.zeros((nb_child * R, nb * R))
        for c in range(nb_child):
            step[c * R:(c + 1) * R, (c // 2) * R:(c // 2 + 1) * R] = E[c % 2].T
        downs.append(downs[-1] @ step)
    for l, nb in enumerate(levels):
        h = np.pi / nb
        nodes = (np.arange(nb)[:, None] + 0.5) * h + 0.5 * h * cheb_nodes()[None, :]
        T = np.zeros((nb * R, nb * R))
        top = l == len(levels) - 1
        for b in range(nb):
            for c in interaction_list(nb, b, top):
                ph, tj = nodes[b][:, None], nodes[c][None, :]
                T[b * R:(b + 1) * R, c * R:(c + 1) * R] = 1.0 / (
                    4.0 * np.sin(0.5 * (ph + tj)) * np.sin(0.5 * (ph - tj)))
        F += downs[l] @ T @ U[l]
    return F


@pytest.mark.parametrize("n", [256, 1024, 4096])
@pytest.mark.parametrize("kind", ["dense_v", "self_loop"])
def test_multilevel_far_field_matches_the_far_part_of_w(n, kind):
    v, rho = (random_unit_v(n, seed=1), 2.0) if kind == "dense_v" else (self_loop_v(n, 0), -0.5)
    plan = cauchy.make_plan(n, v, rho)
    W = cauchy.cauchy_rows(plan, np.arange(n))
    P, _, Q, src_leaf, tgt_leaf = far_field_factors(plan)
    approx = Q @ (multilevel_far_operator(n) @ P)
    far = (tgt_leaf[:, None] >= 0) & (np.abs(tgt_leaf[:, None] - src_leaf[None, :]) >= 2)
    exact = np.where(far, W, 0.0)
    rel = np.linalg.norm(approx - exact, axis=1) / np.linalg.norm(W, axis=1)
    assert rel.max() < 1e-8, rel.max()


def test_multilevel_lists_cover_each_far_leaf_pair_once():
    """Every (target leaf, source leaf) pair at least one leaf apart meets through exactly one
    interaction-list entry over the levels, and no nearer pair does."""
    for nleaf in (4, 16, 64, 256):
        levels = []
        nb = nleaf
        while nb >= 4:
            levels.append(nb)
            nb //= 2
        count = np.zeros((nleaf, nleaf), dtype=int)
        for l, nb in enumerate(levels):
            top = l == len(levels) - 1
            for b in range(nb):
                for c in interaction_list(nb, b, top):
                    count[b << l:(b + 1) << l, c << l:(c + 1) << l] += 1
        i, j = np.meshgrid(np.arange(nleaf), np.arange(nleaf), indexing="ij")
        assert np.array_equal(count, (np.abs(i - j) >= 2).astype(int)), nleaf


def test_reexpansion_is_exact_for_the_parent_basis():
    """M2M loses nothing: the parent's basis restricted to a child is reproduced by the child's
    interpolant (a polynomial of the same degree)."""
    E = child_reexpansion()
    t = cheb_nodes()
    u = np.linspace(-1, 1, 33)
    for k in (0, 1):
        x_parent = (u + 2 * k - 1) / 2.0          # child's [-1, 1] mapped into the parent
        direct = lagrange(x_parent)               # S_a^parent at those points
        via_child = lagrange(u) @ E[k].T          # child's basis times re-expansion
        assert np.abs(direct - via_child).max() < 1e-11
