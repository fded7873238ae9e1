"""The fast form of the paper's trigonometric route (Algorithm 1 steps 4-6), checked in FP64 on
the host against the oracle's direct route.

The GPU kernel replaces the route's three dense sums by FFTs. Each step is rebuilt here in
numpy from its definition, without the CUDA code:
- the orthonormal DCT-II from Makhoul's reordering and a complex FFT of half length;
- the DST-I of Lemma 4.3 from a complex FFT of half length on the symmetrised sequence
  u_j = sin(pi j / N)(f_j + f_{N-j}) + (f_j - f_{N-j}) / 2. The even outputs are -Im U_k and
  the odd outputs the prefix sums Re U_0 / 2 + Re U_1 + ... + Re U_k;
- the sine series sum_l c_l sin(l theta) at the root angles (step 6, the NFST) as a type-2
  nonuniform transform. The coefficients are divided by the Fourier transform of a
  Kaiser-Bessel window of 16 grid steps, a DST-I of length 2n puts the series on the grid
  theta_k = pi k / 2n, and each angle sums the 16 nearest grid values times the window.
The route through these steps must match the oracle's route to rounding, and each step must
match its definition."""
import numpy as np
import pytest
import scipy.fft
import scipy.special

from oracle import cauchy, nfst_route
from synthetic import edge_update_v, normal_signals, random_unit_v, self_loop_v

TAPS = 16
BETA = np.pi * np.sqrt((TAPS / 2) ** 2 * 1.5 ** 2 - 0.8)  # Beatty et al. (2005), oversampling 2


def real_dft_half(y):
    """Y_k = sum_j y_j exp(-2 pi i j k / N), k = 0..N/2, from one complex FFT of length N/2."""
    N = y.size
    L = N // 2
    Z = np.fft.fft(y[0::2] + 1j * y[1::2])
    k = np.arange(L + 1)
    zk, zm = Z[k % L], np.conj(Z[(L - k) % L])
    return (zk + zm) / 2 + np.exp(-2j * np.pi * k / N) * (zk - zm) / 2j


def dst1_fast(f):
    """F_k = sum_{j=1}^{N-1} f_j sin(pi j k / N), k = 0..N (f_0 ignored)."""
    N = f.size
    f = f.copy()
    f[0] = 0.0
    j = np.arange(N)
    fr = f[(N - j) % N]
    u = np.sin(np.pi * j / N) * (f + fr) + 0.5 * (f - fr)
    u[0] = 0.0
    U = real_dft_half(u)
    F = np.zeros(N + 1)
    F[0::2] = -U.imag
    F[1::2] = np.cumsum(U.real[:N // 2]) - U.real[0] / 2
    return F


def dct2_fast(x):
    n = x.size
    v = np.concatenate([x[0::2], x[1::2][::-1]])
    V = real_dft_half(v)
    k = np.arange(n // 2 + 1)
    Q = np.exp(-1j * np.pi * k / (2 * n)) * V
    X = np.empty(n)
    X[k] = Q.real
    X[n - k[1:]] = -Q.imag[1:]
    X *= np.sqrt(2.0 / n)
    X[0] /= np.sqrt(2.0)
    return X


def window(x, alpha):
    t = 1.0 - (x / alpha) ** 2
    return np.where(t > 0, scipy.special.i0(BETA * np.sqrt(np.maximum(t, 0.0))), 0.0)


def window_hat(xi, alpha):
    q = np.sqrt(BETA ** 2 - (alpha * xi) ** 2)
    return 2.0 * alpha * np.sinh(q) / q


def sine_series_fast(c, theta, n):
    """sum_{l=1}^{n-1} c_l sin(l theta) (c indexed by l = 0..n-1, c_0 unused) at every angle."""
    hg = np.pi / (2 * n)
    alpha = TAPS * hg / 2
    d = np.zeros(2 * n)
    l = np.arange(1, n)
    d[1:n] = c[1:] * hg / window_hat(l, alpha)
    G = dst1_fast(d)                                   # G_k, k = 0..2n
    k0 = np.ceil(theta / hg - TAPS / 2).astype(int)
    ks = k0[:, None] + np.arange(TAPS)[None, :]
    idx = np.where(ks < 0, -ks, np.where(ks > 2 * n, 4 * n - ks, ks))
    sign = np.where((ks < 0) | (ks > 2 * n), -1.0, 1.0)
    return (window(theta[:, None] - ks * hg, alpha) * sign * G[idx]).sum(axis=1)


def route_fast(op, x):
    n = op.n
    znd = np.where(op.deflated, 0.0, op.z)
    y = np.empty((x.shape[0], n))
    for b in range(x.shape[0]):
        sd = dct2_fast(x[b])
        s = znd * sd
        j = np.arange(1, n)
        h = np.zeros(n)
        h[1:] = (-1.0) ** (j + 1) * s[1:] / np.sin(np.pi * j / n)
        c = 2.0 * dst1_fast(h)[:n]
        for r in range(n):
            if op.row_kind[r] == 0:
                y[b, r] = sd[op.row_index[r]]
                continue
            i = op.row_index[r]
            mu, a = op.mu[i], op.a[i]
            if 0.0 < mu < 4.0:
                th = 2.0 * np.arctan2(np.sqrt(mu), np.sqrt(4.0 - mu))
                f = sine_series_fast(c, np.array([th]), n)[0]
                y[b, r] = -a * (s[0] / mu - 0.5 * f / np.sin(n * th))
            else:
                y[b, r] = -a * np.sum(s / (mu - op.lam))
    return y


def test_fast_transforms_match_their_definitions():
    rng = np.random.default_rng(0)
    for n in (16, 64, 1024):
        x = rng.standard_normal(n)
        assert np.abs(dct2_fast(x) - scipy.fft.dct(x, norm="ortho")).max() < 1e-13
        f = rng.standard_normal(n)
        F = dst1_fast(f)
        j = np.arange(1, n)
        direct = np.sin(np.pi * np.outer(np.arange(n + 1), j) / n) @ f[1:]
        assert np.abs(F - direct).max() < 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("n", [16, 128, 1024])
def test_window_sum_matches_the_direct_sine_series(n):
    """The nonuniform sine transform reproduces sum_l c_l sin(l theta) to about 1e-14 of
    sum |c_l| at any angle in (0, pi), including angles within one grid step of 0 and pi."""
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n)
    hg = np.pi / (2 * n)
    theta = np.concatenate([rng.uniform(0, np.pi, 200), [0.3 * hg, np.pi - 0.3 * hg, 7.5 * hg]])
    direct = np.sin(np.outer(theta, np.arange(1, n))) @ c[1:]
    fast = sine_series_fast(c, theta, n)
    assert np.abs(fast - direct).max() < 5e-14 * np.abs(c[1:]).sum()


def test_a_wrong_window_constant_is_caught():
    """Dropping the grid step from the deconvolution (a plausible slip) fails the series check."""
    n = 64
    c = np.random.default_rng(1).standard_normal(n)
    theta = np.linspace(0.1, 3.0, 17)
    direct = np.sin(np.outer(theta, np.arange(1, n))) @ c[1:]
    hg = np.pi / (2 * n)
    wrong = sine_series_fast(c, theta, n) / hg
    assert np.abs(wrong - direct).max() > 1e-3


@pytest.mark.parametrize("n", [16, 64, 256])
def test_fast_route_matches_the_oracle_route(n):
    for v, rho in [(random_unit_v(n, seed=7), 0.7), (random_unit_v(n, seed=8), -0.3),
                   (self_loop_v(n, 0), 2.0), (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
        op = cauchy.make_plan(n, v, rho)
        x = normal_signals(3, n, seed=n)
        same = nfst_route.transform(op, x)
        got = route_fast(op, x)
        rel = np.linalg.norm(got - same, axis=1) / np.linalg.norm(same, axis=1)
        assert rel.max() < 1e-11, (n, rho, rel.max())
