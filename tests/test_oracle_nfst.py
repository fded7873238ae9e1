"""Pins of the oracle's version of the paper's trigonometric route (Algorithm 1 steps 3-7):
Gastinel's identity against the direct rational sum, agreement with the Cauchy-formula oracle
where the route is well conditioned, and planted mistakes."""
import numpy as np
import pytest

from oracle import cauchy, nfst_route
from synthetic import edge_update_v, normal_signals, random_unit_v, self_loop_v


@pytest.mark.parametrize("n", [4, 9, 32, 100])
def test_gastinel_identity_against_the_rational_sum(n):
    rng = np.random.default_rng(n)
    s = rng.standard_normal((3, n - 1))
    c = nfst_route.dst1_coefficients(s)
    poles = np.pi * np.arange(1, n) / n
    # angles well inside the gaps between pole angles, plus near both ends
    theta = np.concatenate([poles[:-1] + 0.37 * np.pi / n, [0.21 * np.pi / n, np.pi - 0.33 * np.pi / n]])
    direct = s @ (1.0 / (np.cos(theta)[None, :] - np.cos(poles)[:, None]))
    series = nfst_route.sine_series(c, theta) / np.sin(n * theta)[None, :]
    assert np.abs(series - direct).max() < 1e-10 * np.abs(direct).max()


def route_conditioning(plan):
    """Smallest |sin(n theta)| over the roots evaluated by the trigonometric series."""
    mu = plan.mu
    inside = (mu > 0) & (mu < 4)
    theta = 2 * np.arctan2(np.sqrt(mu[inside]), np.sqrt(4 - mu[inside]))
    return np.abs(np.sin(plan.n * theta)).min()


@pytest.mark.parametrize("n,v,rho", [(8, random_unit_v(8, seed=3), 0.7), (16, self_loop_v(16, 0), 1.5),
                                     (64, random_unit_v(64, seed=5), 2.0), (128, random_unit_v(128), -0.3),
                                     (40, edge_update_v(40, 19, 20), -0.5), (33, self_loop_v(33, 0), 0.25)])
def test_route_matches_the_cauchy_formula(n, v, rho):
    plan = cauchy.make_plan(n, v, rho)
    x = normal_signals(6, n, seed=n)
    ref = cauchy.transform(plan, x)
    got = nfst_route.transform(plan, x)
    # the quotient by sin(n theta) costs about eps / |sin(n theta)| relative accuracy
    tol = 1e-13 / route_conditioning(plan) * n
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < max(tol, 1e-12), (err.max(), tol)


def test_route_degrades_near_a_pole():
    """A tiny z_j puts a root very close to its pole: the route then loses digits that the
    Cauchy formula (gaps as pole + offset) keeps."""
    import scipy.fft
    n = 64
    errs = []
    for tiny in (1e-2, 1e-5):
        z = np.random.default_rng(2).standard_normal(n)
        z[10] = tiny                       # z = U^T v: a small weight on pole 10
        v = scipy.fft.idct(z, norm="ortho")
        v /= np.linalg.norm(v)
        plan = cauchy.make_plan(n, v, 1.0)
        x = normal_signals(4, n, seed=1)
        errs.append((route_conditioning(plan),
                     np.abs(nfst_route.transform(plan, x) - cauchy.transform(plan, x)).max()))
    (c_far, e_far), (c_near, e_near) = errs
    assert c_near < 1e-7 < c_far
    assert e_near > 100 * e_far  # the route loses digits; the pole + offset form does not


def test_planted_route_mistakes_are_caught(monkeypatch):
    n, v, rho = 32, random_unit_v(32, seed=4), 0.9
    plan = cauchy.make_plan(n, v, rho)
    x = normal_signals(3, n, seed=2)
    ref = cauchy.transform(plan, x)
    orig = nfst_route.dst1_coefficients
    monkeypatch.setattr(nfst_route, "dst1_coefficients", lambda s: orig(s) * 2.0)  # factor of Lemma 4.3
    assert np.abs(nfst_route.transform(plan, x) - ref).max() > 1e-3
    monkeypatch.setattr(nfst_route, "dst1_coefficients", lambda s: orig(np.abs(s)))  # lost signs
    assert np.abs(nfst_route.transform(plan, x) - ref).max() > 1e-3
    monkeypatch.setattr(nfst_route, "dst1_coefficients", orig)
    assert np.abs(nfst_route.transform(plan, x) - ref).max() < 1e-10
