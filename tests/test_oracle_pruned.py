"""Pins of the oracle's pruned transform (Theorem 3.4), each against something
other than the function under test: the Jacobi eigenbasis, SciPy's DCT, the
triangle-inequality bound of the theorem, and the exact transform."""
import numpy as np
import pytest
import scipy.fft

from oracle import cauchy, definition
from synthetic import ar1_signals, edge_update_v, normal_signals, random_unit_v, self_loop_v

CASES = [(32, self_loop_v(32, 0), 0.75), (48, random_unit_v(48, seed=4), -0.3),
         (40, edge_update_v(40, 19, 20), -0.5), (64, self_loop_v(64, 0), 2.0)]


def jacobi_w(n, v, rho):
    """W = X^T U from the Jacobi eigenbasis (O1) and SciPy's orthonormal DCT-II matrix."""
    t = definition.transform_matrix(n, v, rho)  # X^T
    u_t = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)  # U^T
    return t @ u_t.T


@pytest.mark.parametrize("n,v,rho", CASES)
def test_pruned_matches_jacobi_blocks(n, v, rho):
    plan = cauchy.make_plan(n, v, rho)
    w = jacobi_w(n, v, rho)
    x = normal_signals(7, n, seed=n)
    s = scipy.fft.dct(x, type=2, norm="ortho", axis=1)
    for m_out, c_p in [(n // 4, n // 4), (n // 4, n // 2), (n // 2, n), (n, n), (1, 1)]:
        got = cauchy.pruned_transform(plan, x, m_out, c_p)
        want = s[:, :c_p] @ w[:m_out, :c_p].T
        assert np.abs(got - want).max() < 1e-10, (m_out, c_p)


@pytest.mark.parametrize("n,v,rho", CASES)
def test_full_width_pruning_is_exact(n, v, rho):
    plan = cauchy.make_plan(n, v, rho)
    x = ar1_signals(5, n, seed=1)
    full = definition.transform(n, v, rho, x)
    for m_out in (1, n // 8, n // 2, n):
        assert np.abs(cauchy.pruned_transform(plan, x, m_out, n) - full[:, :m_out]).max() < 1e-10


@pytest.mark.parametrize("n,v,rho", CASES)
def test_theorem_3_4_bound(n, v, rho):
    plan = cauchy.make_plan(n, v, rho)
    x = np.concatenate([normal_signals(6, n, seed=2), ar1_signals(6, n, seed=3)])
    full = definition.transform(n, v, rho, x)
    for c_p in (n // 8, n // 4, n // 2):
        pruned = np.zeros_like(full)
        pruned[:, :c_p] = cauchy.pruned_transform(plan, x, c_p, c_p)
        err = np.linalg.norm(full - pruned, axis=1)
        bound = cauchy.pruning_bound(plan, x, c_p)
        assert np.all(err <= bound * (1 + 1e-12) + 1e-13)
        # the error is W [0; s_h] + [0; W_hl s_l] with W orthogonal, so the reverse
        # triangle inequality bounds it from below by | ||s_h|| - ||W_hl s_l|| |
        s = scipy.fft.dct(x, type=2, norm="ortho", axis=1)
        w = jacobi_w(n, v, rho)
        sh = np.linalg.norm(s[:, c_p:], axis=1)
        leak = np.linalg.norm(s[:, :c_p] @ w[c_p:, :c_p].T, axis=1)
        assert np.allclose(bound, sh + leak, rtol=1e-9)
        assert np.all(err >= np.abs(sh - leak) * (1 - 1e-9) - 1e-12)


def test_band_limited_signal_error_is_the_leakage_term():
    n, v, rho = 32, self_loop_v(32, 0), 1.0
    plan = cauchy.make_plan(n, v, rho)
    c_p = 8
    s = np.zeros((3, n))
    s[:, :c_p] = normal_signals(3, c_p, seed=9)
    x = scipy.fft.idct(s, type=2, norm="ortho", axis=1)
    full = definition.transform(n, v, rho, x)
    pruned = np.zeros_like(full)
    pruned[:, :c_p] = cauchy.pruned_transform(plan, x, c_p, c_p)
    err = np.linalg.norm(full - pruned, axis=1)
    w = jacobi_w(n, v, rho)
    leak = np.linalg.norm(s[:, :c_p] @ w[c_p:, :c_p].T, axis=1)
    # with s_h = 0 the error vector is [0; W_hl s_l] exactly
    assert np.allclose(err, leak, rtol=1e-10, atol=1e-13)
    assert np.allclose(cauchy.pruning_bound(plan, x, c_p), leak, rtol=1e-10, atol=1e-13)


def test_planted_block_mistake_is_caught(monkeypatch):
    n, v, rho = 32, random_unit_v(32, seed=4), -0.3
    plan = cauchy.make_plan(n, v, rho)
    w = jacobi_w(n, v, rho)
    x = normal_signals(4, n, seed=5)
    s = scipy.fft.dct(x, type=2, norm="ortho", axis=1)
    want = s[:, :8] @ w[:8, :8].T
    orig = cauchy.cauchy_rows
    # a pruned product that takes the wrong row block (rows shifted by one)
    monkeypatch.setattr(cauchy, "cauchy_rows", lambda p, rows: orig(p, np.asarray(rows) + 1))
    assert np.abs(cauchy.pruned_transform(plan, x, 8, 8) - want).max() > 1e-3


def test_argument_checks():
    plan = cauchy.make_plan(16, self_loop_v(16, 0), 1.0)
    x = normal_signals(2, 16, seed=0)
    for m_out, c_p in [(0, 4), (5, 4), (4, 17)]:
        with pytest.raises(ValueError):
            cauchy.pruned_transform(plan, x, m_out, c_p)
