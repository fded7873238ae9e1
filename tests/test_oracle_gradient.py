"""Pins of the oracle's gradients: central finite differences of the Jacobi
(O1) forward transform, adjoint identities, and planted mistakes."""
import numpy as np
import pytest

from oracle import cauchy, definition, gradient
from synthetic import ar1_signals, edge_update_v, normal_signals, random_unit_v, self_loop_v

CASES = [(8, self_loop_v(8, 0), 1.0), (12, random_unit_v(12, seed=3), -0.3),
         (16, random_unit_v(16, seed=5), 2.0), (16, edge_update_v(16, 7, 8), -0.5),
         (10, self_loop_v(10, 0), 0.0)]


def loss_o1(n, v, rho, x, gw):
    """<gw, y> with y from the Jacobi eigenbasis: its gradient in y is gw."""
    return float(np.sum(gw * definition.transform(n, v, rho, x)))


def fd_grads(n, v, rho, x, gw, h=1e-6):
    d_rho = (loss_o1(n, v, rho + h, x, gw) - loss_o1(n, v, rho - h, x, gw)) / (2 * h)
    d_v = np.empty(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        d_v[j] = (loss_o1(n, v + e, rho, x, gw) - loss_o1(n, v - e, rho, x, gw)) / (2 * h)
    return d_rho, d_v


@pytest.mark.parametrize("n,v,rho", CASES)
def test_parameter_gradients_match_finite_differences(n, v, rho):
    x = normal_signals(5, n, seed=n)
    gw = normal_signals(5, n, seed=n + 100)
    plan = cauchy.make_plan(n, v, rho)
    g_rho, g_v = gradient.parameter_gradients(plan, x, gw)
    f_rho, f_v = fd_grads(n, v, rho, x, gw)
    scale = max(1.0, abs(f_rho))
    assert abs(g_rho - f_rho) < 2e-6 * scale, (g_rho, f_rho)
    assert np.abs(g_v - f_v).max() < 2e-6 * max(1.0, np.abs(f_v).max()), np.abs(g_v - f_v).max()


def test_squared_tail_loss_matches_finite_differences():
    """The differentiable workload's loss: sum of squared coefficients of the upper half."""
    n = 16
    v, rho = random_unit_v(n, seed=9), 2.0
    x = ar1_signals(4, n, seed=2)

    def loss(v_, rho_):
        y = definition.transform(n, v_, rho_, x)
        return float(np.sum(y[:, n // 2:] ** 2))

    plan = cauchy.make_plan(n, v, rho)
    y = cauchy.transform(plan, x)
    gy = np.zeros_like(y)
    gy[:, n // 2:] = 2 * y[:, n // 2:]
    g_rho, g_v = gradient.parameter_gradients(plan, x, gy)
    h = 1e-6
    f_rho = (loss(v, rho + h) - loss(v, rho - h)) / (2 * h)
    f_v = np.array([(loss(v + h * e, rho) - loss(v - h * e, rho)) / (2 * h) for e in np.eye(n)])
    assert abs(g_rho - f_rho) < 2e-6 * max(1, abs(f_rho))
    assert np.abs(g_v - f_v).max() < 2e-6 * max(1, np.abs(f_v).max())
    # the signal gradient by finite differences of the same loss
    gx = gradient.backward_x(plan, gy)
    fx = np.empty_like(x)
    for b in range(x.shape[0]):
        for j in range(n):
            xp, xm = x.copy(), x.copy()
            xp[b, j] += h
            xm[b, j] -= h
            yp = definition.transform(n, v, rho, xp)
            ym = definition.transform(n, v, rho, xm)
            fx[b, j] = (np.sum(yp[:, n // 2:] ** 2) - np.sum(ym[:, n // 2:] ** 2)) / (2 * h)
    assert np.abs(gx - fx).max() < 1e-6 * max(1, np.abs(fx).max())


@pytest.mark.parametrize("n,v,rho", CASES)
def test_backward_x_is_the_adjoint_and_the_inverse(n, v, rho):
    plan = cauchy.make_plan(n, v, rho)
    x = normal_signals(6, n, seed=1)
    g = normal_signals(6, n, seed=2)
    y = cauchy.transform(plan, x)
    gx = gradient.backward_x(plan, g)
    assert abs(np.sum(y * g) - np.sum(x * gx)) < 1e-11 * np.abs(y * g).sum()
    assert np.abs(gradient.backward_x(plan, y) - x).max() < 1e-12


def test_w_of_roots_is_minus_a_over_rho():
    n = 24
    plan = cauchy.make_plan(n, random_unit_v(n, seed=7), 0.7)
    w = cauchy.transform_matrix(plan) @ plan.v
    roots = plan.row_kind == 1
    a = plan.a[plan.row_index[roots]]
    assert np.abs(w[roots] + a / plan.rho).max() < 1e-12


def test_planted_gradient_mistakes_are_caught(monkeypatch):
    n, v, rho = 12, random_unit_v(12, seed=3), -0.3
    x = normal_signals(3, n, seed=4)
    gw = normal_signals(3, n, seed=5)
    f_rho, f_v = fd_grads(n, v, rho, x, gw)
    plan = cauchy.make_plan(n, v, rho)
    orig_k = gradient.cauchy_k

    def caught():
        g_rho, g_v = gradient.parameter_gradients(plan, x, gw)
        return abs(g_rho - f_rho) > 1e-4 or np.abs(g_v - f_v).max() > 1e-4

    monkeypatch.setattr(gradient, "cauchy_k", lambda p: orig_k(p).T)  # transposed K
    assert caught()
    monkeypatch.setattr(gradient, "cauchy_k", lambda p: -orig_k(p))   # sign of the gaps
    assert caught()
    monkeypatch.setattr(gradient, "cauchy_k", orig_k)
    assert not caught()
