"""Band matrices and their LU factorization without pivoting (oracle, plain CPU code).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

The coarse problem of Eq. 9 is solved with A_0 = P_0^T DF P_0 in band storage: row i holds the
entries (i, i - b + d) for d = 0 .. 2b at position i (2b + 1) + d (entries outside the matrix are
zero).  Gaussian elimination without row exchanges keeps every factor inside the band, so the
factors use the same storage: d < b the multipliers of the unit lower factor L, d = b the
reciprocal pivot 1 / U_ii, d > b the entries of U above the diagonal.  This is the textbook
elimination written out step by step (for k = 0 .. n-1: l_ik = a_ik / a_kk, a_ij -= l_ik a_kj for
the rows and columns within the band), in FP64.
"""
from __future__ import annotations

import numpy as np


def band_to_dense(band: np.ndarray) -> np.ndarray:
    """Dense n x n matrix of a band array [n, 2b + 1]."""
    n, w = band.shape
    b = (w - 1) // 2
    A = np.zeros((n, n))
    for i in range(n):
        for d in range(w):
            j = i - b + d
            if 0 <= j < n:
                A[i, j] = band[i, d]
    return A


def dense_to_band(A: np.ndarray, b: int) -> np.ndarray:
    """Band array [n, 2b + 1] of the entries of A with |i - j| <= b."""
    n = A.shape[0]
    band = np.zeros((n, 2 * b + 1))
    for i in range(n):
        for d in range(2 * b + 1):
            j = i - b + d
            if 0 <= j < n:
                band[i, d] = A[i, j]
    return band


def lu_nopivot(band: np.ndarray) -> np.ndarray:
    """Factors of A = L U (no pivoting) in the band layout described above; raises
    ZeroDivisionError on a zero pivot."""
    n, w = band.shape
    b = (w - 1) // 2
    A = band_to_dense(band)
    for k in range(n):
        piv = A[k, k]
        if piv == 0.0 or not np.isfinite(piv):
            raise ZeroDivisionError(f"pivot {k} is {piv}")
        hi = min(n, k + b + 1)
        A[k + 1:hi, k] /= piv
        A[k + 1:hi, k + 1:hi] -= np.outer(A[k + 1:hi, k], A[k, k + 1:hi])
    F = dense_to_band(A, b)
    F[:, b] = 1.0 / np.diag(A)
    return F


def factors_dense(F: np.ndarray):
    """(L, U) as dense matrices from the band factors."""
    n, w = F.shape
    b = (w - 1) // 2
    M = band_to_dense(F)
    L = np.tril(M, -1) + np.eye(n)
    U = np.triu(M, 1) + np.diag(1.0 / F[:, b])
    return L, U
