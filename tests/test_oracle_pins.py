"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself or with the CUDA path:
closed forms (DCT-II, path eigenvalues, DST-VII, the n = 2 quadratic),
invariants (Lemma 4.1 interlacing, the secular equation, the trace identity,
orthonormality, v^T x_i = -a_i / rho), brute force in 50-digit arithmetic at
n <= 8, the definition-based O1 against the formula-based O2, and Table 1's
printed accuracy. A final test plants mistakes in the oracle and checks that
the pins catch them.
"""
import os

import numpy as np
import pytest

from oracle import cauchy, common, definition
from oracle._native import jacobi_eigh
from synthetic import ar1_signals, edge_update_v, normal_signals, random_unit_v, self_loop_v

EPS = np.finfo(np.float64).eps

CASES = [
    # (n, v, rho) — self-loops, edge updates (end, interior, central), dense v, both signs
    (2, random_unit_v(2, seed=5), 0.7),
    (3, self_loop_v(3, 0), 1.0),
    (5, edge_update_v(5, 1, 2), -0.4),
    (8, self_loop_v(8, 0), 1.5),
    (8, edge_update_v(8, 3, 4), -0.5),
    (16, random_unit_v(16), 2.0),
    (16, random_unit_v(16), -0.3),
    (31, edge_update_v(31, 2, 4), 1.5),
    (64, self_loop_v(64, 0), 0.5),
    (64, edge_update_v(64, 31, 32), -0.5),
    (64, random_unit_v(64), -0.3),
]


def dst7_matrix(n):
    """Closed-form DST-VII: row k = 2/sqrt(2n+1) sin(pi (2k+1)(j+1)/(2n+1))."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return 2.0 / np.sqrt(2 * n + 1) * np.sin(np.pi * (2 * k + 1) * (j + 1) / (2 * n + 1))


# ---------------------------------------------------------------- path graph, DCT-II

@pytest.mark.parametrize("n", [2, 3, 7, 16, 64])
def test_path_eigenvalues_match_jacobi_and_cosine_form(n):
    lam = common.path_eigenvalues(n)
    w, _ = jacobi_eigh(definition.path_laplacian(n))
    assert np.allclose(lam, w, atol=1e-13, rtol=0)
    assert np.allclose(lam, 2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n), atol=1e-14, rtol=0)
    assert lam[0] == 0.0 and np.all(np.diff(lam) > 0)


@pytest.mark.parametrize("n", [2, 5, 8, 64, 100])
def test_dct2_basis_diagonalises_path_laplacian(n):
    U = common.dct2_basis(n)
    L = definition.path_laplacian(n)
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-13
    assert np.abs(L @ U - U * common.path_eigenvalues(n)[None, :]).max() < 1e-13
    assert np.all(U[0, :] > 0)  # standard DCT-II sign: first sample positive


@pytest.mark.parametrize("n", [4, 9, 64, 257])
def test_dct2_matches_scipy_orthonormal_dct(n):
    scipy_fft = pytest.importorskip("scipy.fft")
    x = normal_signals(5, n, seed=11)
    assert np.abs(common.dct2(x) - scipy_fft.dct(x, type=2, norm="ortho", axis=-1)).max() < 1e-12


def test_pole_differences_product_form():
    n = 16384
    j = np.array([1, 2, 100, 8000, 16383])
    p = np.array([0, 1, 99, 8001, 16382])
    d = common.pole_differences(n, j, p)
    lam = common.path_eigenvalues(n)
    # agrees with the plain difference where that difference has no cancellation
    assert abs(d[0] - (lam[1] - lam[0])) <= 4 * EPS * lam[1]
    # and is accurate where the plain difference cancels (exact: 2 sin(pi (j+p)/2n) ... )
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for jj, pp, dd in zip(j, p, d):
        exact = 4 * mp.sin(mp.pi * jj / (2 * n)) ** 2 - 4 * mp.sin(mp.pi * pp / (2 * n)) ** 2
        assert abs(float(exact) - dd) <= 8 * EPS * abs(float(exact))


# ---------------------------------------------------------------- z = U^T v

@pytest.mark.parametrize("n", [8, 64, 1000])
def test_z_closed_forms(n):
    k = np.arange(n)
    c = np.where(k == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    # self-loop at vertex 0: z_k = c_k cos(pi k / 2n)
    p = cauchy.make_plan(n, self_loop_v(n, 0), 1.0)
    assert np.abs(p.z - c * np.cos(np.pi * k / (2 * n))).max() < 1e-14
    # edge (i, i+1): z_k = 2 c_k sin(pi k (i+1)/n) sin(pi k / 2n)
    i = n // 3
    p = cauchy.make_plan(n, edge_update_v(n, i, i + 1), 0.5)
    m = (k * (i + 1)) % (2 * n)  # reduce the phase exactly before the sine
    ref = 2 * c * np.sin(np.pi * m / n) * np.sin(np.pi * k / (2 * n))
    assert np.abs(p.z - ref).max() < 1e-14
    # Parseval for U^T
    v = random_unit_v(n, seed=3) * 1.7
    p = cauchy.make_plan(n, v, 0.5)
    assert abs(np.linalg.norm(p.z) - 1.7) < 1e-13


def test_structural_zeros_are_deflated():
    n = 64
    p = cauchy.make_plan(n, edge_update_v(n, n // 2 - 1, n // 2), -0.5)
    # central edge: z_k = 0 for all even k (including the DC term)
    assert np.array_equal(p.deflated, np.arange(n) % 2 == 0)
    p = cauchy.make_plan(n, edge_update_v(n, 5, 6), 1.0)
    assert p.deflated[0]                      # constant vector stays in the kernel
    p = cauchy.make_plan(n, random_unit_v(n), 1.0)
    assert not p.deflated.any()
    p = cauchy.make_plan(n, random_unit_v(n), 0.0)
    assert p.deflated.all()                   # rho = 0 leaves the DCT unchanged


# ---------------------------------------------------------------- secular roots

@pytest.mark.parametrize("case", range(len(CASES)))
def test_roots_interlace_and_solve_secular_equation(case):
    n, v, rho = CASES[case]
    p = cauchy.make_plan(n, v, rho)
    mu = p.mu
    lam_nd = p.lam[p.poles]
    K = p.poles.size
    # Lemma 4.1 (and its mirror for rho < 0)
    if rho > 0:
        assert np.all(mu > lam_nd)
        assert np.all(mu[:-1] < lam_nd[1:])
    else:
        assert np.all(mu < lam_nd)
        assert np.all(mu[1:] > lam_nd[:-1])
    # trace identity: sum mu - sum lambda_nd = rho ||z_nd||^2 = rho ||v||^2 (up to deflated mass)
    assert abs(mu.sum() - lam_nd.sum() - rho * np.sum(p.z[p.poles] ** 2)) < 1e-12 * max(1, K)
    # each mu_i is an eigenvalue of the dense L: det(L - mu I) changes sign across it
    L = definition.updated_laplacian(n, v, rho)
    w, _ = jacobi_eigh(L)
    assert np.abs(np.sort(w) - p.eigenvalues).max() < 1e-12


@pytest.mark.parametrize("n", [3, 8, 64, 513])
def test_unit_self_loop_eigenvalues_are_dst7(n):
    p = cauchy.make_plan(n, self_loop_v(n, 0), 1.0)
    ref = 2.0 - 2.0 * np.cos(np.pi * (2 * np.arange(n) + 1) / (2 * n + 1))
    assert np.abs(p.eigenvalues - ref).max() < 1e-13


def test_n2_quadratic_closed_form():
    v = np.array([0.6, -0.8])
    rho = 1.3
    L = definition.updated_laplacian(2, v, rho)
    tr, det = np.trace(L), np.linalg.det(L)
    disc = np.sqrt(tr * tr / 4 - det)
    ref = np.array([tr / 2 - disc, tr / 2 + disc])
    p = cauchy.make_plan(2, v, rho)
    assert np.abs(p.eigenvalues - ref).max() < 1e-14


# ---------------------------------------------------------------- eigenvectors / transform

@pytest.mark.parametrize("case", range(len(CASES)))
def test_transform_is_orthonormal_eigenbasis(case):
    n, v, rho = CASES[case]
    p = cauchy.make_plan(n, v, rho)
    T = cauchy.transform_matrix(p)
    L = definition.updated_laplacian(n, v, rho)
    assert np.abs(T @ T.T - np.eye(n)).max() < 1e-13
    assert np.abs(L @ T.T - T.T * p.eigenvalues[None, :]).max() < 1e-13
    x = normal_signals(7, n, seed=2)
    y = x @ T.T
    assert np.abs(np.linalg.norm(y, axis=1) - np.linalg.norm(x, axis=1)).max() < 1e-12


@pytest.mark.parametrize("case", range(len(CASES)))
def test_v_projection_identity(case):
    """v^T x_i = -a_i sum_j z_j^2/(mu_i - lambda_j) = -a_i / rho (Lemma 4.2 + secular eq.)."""
    n, v, rho = CASES[case]
    p = cauchy.make_plan(n, v, rho)
    T = cauchy.transform_matrix(p)
    root_rows = np.nonzero(p.row_kind == 1)[0]
    proj = T[root_rows] @ v
    assert np.abs(proj - (-p.a[p.row_index[root_rows]] / rho)).max() < 1e-11


@pytest.mark.parametrize("case", range(len(CASES)))
def test_definition_oracle_matches_cauchy_oracle(case):
    n, v, rho = CASES[case]
    T1 = definition.transform_matrix(n, v, rho)
    p = cauchy.make_plan(n, v, rho)
    T2 = cauchy.transform_matrix(p)
    gap = np.min(np.diff(p.eigenvalues)) if n > 1 else 1.0
    # eigenvectors are determined to about (residual / eigen-gap) (Davis-Kahan)
    tol = 1e-13 + 64 * EPS * 4.0 * max(1.0, abs(rho)) / gap
    assert np.abs(T1 - T2).max() < tol


@pytest.mark.parametrize("n", [4, 16, 64])
def test_rho_zero_is_orthonormal_dct2(n):
    T = cauchy.transform_matrix(cauchy.make_plan(n, random_unit_v(n), 0.0))
    assert np.abs(T - common.dct2_basis(n).T).max() < 1e-15
    T1 = definition.transform_matrix(n, random_unit_v(n), 0.0)
    assert np.abs(T1 - common.dct2_basis(n).T).max() < 1e-12


def test_unit_self_loop_at_vertex0_is_dst7_with_signs():
    """The FP64 n=64 configuration: rho = 1, v = e_0 gives the DST-VII exactly."""
    n = 64
    ref = dst7_matrix(n)
    T2 = cauchy.transform_matrix(cauchy.make_plan(n, self_loop_v(n, 0), 1.0))
    T1 = definition.transform_matrix(n, self_loop_v(n, 0), 1.0)
    assert np.abs(T2 - ref).max() < 1e-14
    assert np.abs(T1 - ref).max() < 1e-12
    x = normal_signals(1024, n, seed=0)
    assert np.abs(x @ T2.T - x @ ref.T).max() < 1e-12


def test_central_edge_keeps_even_dct_rows():
    n = 32
    p = cauchy.make_plan(n, edge_update_v(n, n // 2 - 1, n // 2), -0.5)
    x = normal_signals(9, n, seed=4)
    y = cauchy.transform(p, x)
    s = common.dct2(x)
    for r in np.nonzero(p.row_kind == 0)[0]:
        j = p.row_index[r]
        assert j % 2 == 0
        assert np.abs(y[:, r] - s[:, j]).max() < 1e-15
    # the DC coefficient of an edge update is unchanged and comes first
    assert p.row_kind[0] == 0 and p.row_index[0] == 0


def test_bruteforce_50_digits_small_n():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for n, v, rho in [(2, [0.6, -0.8], 1.3), (4, [1, 0, 0, 0], 1.0), (5, [0, 1, -1, 0, 0], -0.4),
                      (6, list(random_unit_v(6, seed=9)), 2.5), (8, list(random_unit_v(8, seed=7)), -0.3)]:
        v = np.asarray(v, dtype=np.float64)
        A = mp.matrix(n, n)
        for i in range(n):
            for j in range(n):
                A[i, j] = mp.mpf(rho) * mp.mpf(v[i]) * mp.mpf(v[j])
        for i in range(n - 1):
            A[i, i] += 1
            A[i + 1, i + 1] += 1
            A[i, i + 1] -= 1
            A[i + 1, i] -= 1
        E, Q = mp.eigsy(A)
        order = sorted(range(n), key=lambda i: E[i])
        Uhp = mp.matrix(n, n)
        for j in range(n):
            for k in range(n):
                c = mp.sqrt(mp.mpf(1) / n) if k == 0 else mp.sqrt(mp.mpf(2) / n)
                Uhp[j, k] = c * mp.cos(mp.pi * k * (2 * j + 1) / (2 * n))
        p = cauchy.make_plan(n, v, rho)
        T = cauchy.transform_matrix(p)
        for r, i in enumerate(order):
            assert abs(float(E[i]) - p.eigenvalues[r]) < 1e-14
            q = [Q[jj, i] for jj in range(n)]
            # orient the 50-digit vector with the same pairing rule as the oracle
            if p.row_kind[r] == 0:
                pole = p.row_index[r]
            else:
                pole = p.poles[p.row_index[r]]
            proj = sum(Uhp[jj, pole] * q[jj] for jj in range(n))
            sgn = 1 if proj > 0 else -1
            for jj in range(n):
                assert abs(float(sgn * q[jj]) - T[r, jj]) < 1e-14


def _read_table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_snr.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[2]), float(r[3])) for r in rows}


@pytest.mark.slow
def test_fp64_formula_is_at_least_as_accurate_as_table1():
    """O2 against NMVP on AR(0.99) signals reaches at least the SNR the paper prints."""
    table = _read_table1()
    for n in (8, 16, 32, 64, 128, 256):
        alpha = 1.5
        updates = [(edge_update_v(n, 1, 2), alpha), (self_loop_v(n, 0), alpha),
                   (edge_update_v(n, 2, 4), alpha)]
        x = ar1_signals(64, n, 0.99, seed=0)
        for (v, rho), printed in zip(updates, table[n]):
            y1 = definition.transform(n, v, rho, x)
            y2 = cauchy.transform(cauchy.make_plan(n, v, rho), x)
            snr = np.mean(10 * np.log10(np.sum(y1 ** 2, 1) / np.sum((y1 - y2) ** 2, 1)))
            assert snr >= printed, (n, printed, snr)


def test_large_n_sampled_rows_are_consistent():
    """At n = 4096 the sampled-root plan agrees with the full plan on those rows."""
    n = 4096
    v = random_unit_v(n)
    rows = [0, 1, 2, 1000, 2047, 4094, 4095]
    full = cauchy.make_plan(n, v, 2.0)
    part = cauchy.make_plan(n, v, 2.0, roots=rows)
    assert np.array_equal(full.tau[rows], part.tau[rows])
    x = normal_signals(3, n, seed=1)
    y = cauchy.transform(part, x, rows=rows)
    T = cauchy.cauchy_rows(full, rows)
    s = common.dct2(x)
    assert np.abs(y - s @ T.T).max() < 1e-13
    # rows are unit vectors
    assert np.abs(np.linalg.norm(T, axis=1) - 1).max() < 1e-12


# ---------------------------------------------------------------- planted mistakes

def _pins_hold(n, v, rho):
    p = cauchy.make_plan(n, v, rho)
    T = cauchy.transform_matrix(p)
    L = definition.updated_laplacian(n, v, rho)
    ok = np.abs(T @ T.T - np.eye(n)).max() < 1e-12
    ok &= np.abs(L @ T.T - T.T * p.eigenvalues[None, :]).max() < 1e-12
    T1 = definition.transform_matrix(n, v, rho)
    ok &= np.abs(T1 - T).max() < 1e-9
    if np.array_equal(v, self_loop_v(n, 0)) and rho == 1.0:
        ok &= np.abs(T - dst7_matrix(n)).max() < 1e-12
    return bool(ok)


def test_planted_mistakes_are_caught(monkeypatch):
    n = 16
    cases = [(n, self_loop_v(n, 0), 1.0), (n, random_unit_v(n), -0.3), (n, edge_update_v(n, 3, 4), 0.8)]
    assert all(_pins_hold(*c) for c in cases)

    orig_rows = cauchy.cauchy_rows
    orig_lam = cauchy.path_eigenvalues
    orig_pd = cauchy.pole_differences
    orig_dct = cauchy.dct2

    mutants = {
        "dropped z factor": lambda: monkeypatch.setattr(
            cauchy, "cauchy_rows",
            lambda p, rows: orig_rows(p, rows) / np.where(p.z == 0, 1, p.z)[None, :]),
        "sign of a flipped": lambda: monkeypatch.setattr(
            cauchy, "cauchy_rows", lambda p, rows: -orig_rows(p, rows)),
        "transposed operand": lambda: monkeypatch.setattr(
            cauchy, "transform_matrix",
            lambda p: (orig_rows(p, np.arange(p.n)) @ common.dct2_basis(p.n).T).T),
        "eigenvalue index off by one": lambda: monkeypatch.setattr(
            cauchy, "path_eigenvalues", lambda n: orig_lam(n + 1)),
        "pole difference sign": lambda: monkeypatch.setattr(
            cauchy, "pole_differences", lambda n, r, c: -orig_pd(n, r, c)),
        "unnormalised DCT": lambda: monkeypatch.setattr(
            cauchy, "dct2", lambda x: orig_dct(x) * 2.0),
    }
    for name, plant in mutants.items():
        with monkeypatch.context() as m:  # noqa: F841
            plant()
            try:
                held = all(_pins_hold(*c) for c in cases)
            except Exception:
                held = False
            monkeypatch.undo()
        assert not held, f"planted mistake not caught: {name}"
