"""Quantities of the unperturbed path graph used by both oracles.

Test infrastructure only: the product path never imports this package.

The path graph on n vertices has the Laplacian L~ of Def. 2.2 (diagonal
[1, 2, ..., 2, 1], off-diagonals -1). Its GFT basis is the orthonormal DCT-II
(Sec. 4.2, "the product with U^T is in O(n log n) via DCT") and its eigenvalues
are lambda_k = 2 - 2 cos(pi k / n) (Sec. 4.2.2 uses 1 - lambda_{k+1}/2 as the
roots of the Chebyshev polynomial U_{n-1}).
"""
from __future__ import annotations

import numpy as np


def path_eigenvalues(n: int) -> np.ndarray:
    """lambda_k = 4 sin^2(pi k / 2n) = 2 - 2 cos(pi k / n), k = 0..n-1, ascending."""
    k = np.arange(n, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2


def pole_differences(n: int, rows, cols) -> np.ndarray:
    """lambda_rows - lambda_cols without cancellation.

    sin^2(A) - sin^2(B) = sin(A + B) sin(A - B), so
    lambda_j - lambda_p = 4 sin(pi (j + p) / 2n) sin(pi (j - p) / 2n).
    The first factor is taken as sin(pi m / 2n) with m = min(j + p, 2n - j - p)
    (same value, argument at most pi/2), so near j + p = 2n it is not the sine
    of a rounded number close to pi.
    """
    j = np.asarray(rows, dtype=np.int64)
    p = np.asarray(cols, dtype=np.int64)
    m = j + p
    m = np.minimum(m, 2 * n - m).astype(np.float64)
    return 4.0 * np.sin(np.pi * m / (2.0 * n)) * np.sin(np.pi * (j - p).astype(np.float64) / (2.0 * n))


def dct2_basis(n: int, cols=None) -> np.ndarray:
    """U[j, k] = c_k cos(pi k (2j + 1) / 2n), c_0 = sqrt(1/n), c_k = sqrt(2/n).

    Column k is the k-th eigenvector of L~. The phase k(2j+1) is reduced
    modulo 4n in integers before the cosine so large n loses no accuracy.
    ``cols`` selects a subset of columns (default: all).
    """
    k = np.arange(n, dtype=np.int64) if cols is None else np.asarray(cols, dtype=np.int64)
    j = np.arange(n, dtype=np.int64)
    m = (np.outer(2 * j + 1, k)) % (4 * n)
    c = np.where(k == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    return np.cos(np.pi * m / (2.0 * n)) * c[None, :]


def dct2(x: np.ndarray, block: int = 2048) -> np.ndarray:
    """Orthonormal DCT-II of each row of x by the direct O(n^2) sum s = x U."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    n = x.shape[1]
    out = np.empty_like(x)
    for k0 in range(0, n, block):
        cols = np.arange(k0, min(n, k0 + block))
        out[:, cols] = x @ dct2_basis(n, cols)
    return out


def deflation_mask(z: np.ndarray, rho: float) -> np.ndarray:
    """Indices whose z_j is treated as zero (Sec. 4: "we can apply deflation first").

    The paper fixes no tolerance. Reading used here: deflate j when
    |rho| |z_j| ||z|| <= 2^-48 max(1, |rho| ||z||^2, 4), i.e. when the part of
    rho v v^T that couples u_j to the rest is below about 16 units in the last
    place of ||L|| (4 bounds lambda_max). rho = 0 deflates every index.
    """
    z = np.asarray(z, dtype=np.float64)
    nz = np.linalg.norm(z)
    scale = max(1.0, abs(rho) * nz * nz, 4.0)
    return abs(rho) * np.abs(z) * nz <= 2.0 ** -48 * scale
