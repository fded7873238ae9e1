"""Oracle O1: the DCT+ transform by its definition (Def. 2.2, Def. 2.3).

Test infrastructure only; the product path never imports it.

Build the dense generalised Laplacian L = L~ + rho v v^T, diagonalise it with
cyclic Jacobi rotations (``jacobi.c``), sort the eigenpairs by ascending
eigenvalue, orient each eigenvector, and apply X^T to the signals with a
plain matrix product (the paper's NMVP comparator, Sec. 5).

Orientation (the paper leaves the sign of a_i open, Theorem 3.1): an
eigenvector that is a deflated DCT vector u_j (z_j ~ 0, Sec. 4) is oriented
with <u_j, x> > 0; the remaining eigenvectors, in ascending order, are paired
with the non-deflated poles in ascending order and oriented so that
<u_pole, x> > 0. Deflation uses the same reading as O2
(``common.deflation_mask``).
"""
from __future__ import annotations

import numpy as np

from ._native import jacobi_eigh
from .common import deflation_mask, dct2_basis


def path_laplacian(n: int) -> np.ndarray:
    """L~ = D - W for the unweighted path graph on n vertices (Def. 2.2, no self-loops)."""
    L = np.zeros((n, n))
    for i in range(n - 1):
        L[i, i] += 1.0
        L[i + 1, i + 1] += 1.0
        L[i, i + 1] -= 1.0
        L[i + 1, i] -= 1.0
    return L


def updated_laplacian(n: int, v, rho: float) -> np.ndarray:
    """L(v, rho) = L~ + rho v v^T (Def. 2.3)."""
    v = np.asarray(v, dtype=np.float64)
    return path_laplacian(n) + rho * np.outer(v, v)


def gft(n: int, v, rho: float):
    """Return (eigenvalues ascending, X) with X[:, i] the oriented i-th eigenvector of L(v, rho)."""
    L = updated_laplacian(n, v, rho)
    w, X = jacobi_eigh(L)
    U = dct2_basis(n)
    z = U.T @ np.asarray(v, dtype=np.float64)
    deflated = deflation_mask(z, rho)
    C = U.T @ X                       # C[k, i] = <u_k, x_i>
    is_defl_vec = np.zeros(n, dtype=bool)
    pair = np.empty(n, dtype=np.int64)
    for j in np.nonzero(deflated)[0]:
        cand = np.where(is_defl_vec, -1.0, np.abs(C[j, :]))
        i = int(np.argmax(cand))
        is_defl_vec[i] = True
        pair[i] = j
    rest = np.nonzero(~is_defl_vec)[0]          # ascending eigenvalue order
    nd_poles = np.nonzero(~deflated)[0]         # ascending pole order
    pair[rest] = nd_poles
    signs = np.sign(C[pair, np.arange(n)])
    signs[signs == 0] = 1.0
    return w, X * signs[None, :]


def transform_matrix(n: int, v, rho: float) -> np.ndarray:
    """T = X^T: y = T x gives the GFT coefficients in ascending eigenvalue order."""
    _, X = gft(n, v, rho)
    return X.T


def transform(n: int, v, rho: float, x) -> np.ndarray:
    """NMVP: y = X^T x for each row of x."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return x @ transform_matrix(n, v, rho).T
