"""Pins of the oracle's band LU without pivoting (oracle/banded.py) against facts outside it:
the factors reproduce A = L U, they coincide with scipy's partial-pivoting LU on matrices that
are diagonally dominant by columns (where partial pivoting never exchanges rows), the band stays
free of fill, and a hand-computed 3 x 3 case."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import banded as B


def column_dominant_band(n, b, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - b), min(n, i + b + 1)):
            A[i, j] = rng.uniform(-1.0, 1.0)
    # strictly diagonally dominant by columns: partial pivoting keeps the diagonal pivot
    for j in range(n):
        A[j, j] = np.sign(A[j, j] or 1.0) * (np.abs(A[:, j]).sum() + 1.0)
    return A


def test_hand_computed_3x3():
    A = np.array([[4.0, 2.0, 0.0], [2.0, 5.0, 1.0], [0.0, 1.0, 3.0]])
    F = B.lu_nopivot(B.dense_to_band(A, 1))
    # l10 = 1/2, u11 = 5 - 1 = 4, l21 = 1/4, u22 = 3 - 1/4
    np.testing.assert_allclose(F[1, 0], 0.5, rtol=0, atol=0)
    np.testing.assert_allclose(F[2, 0], 0.25, rtol=0, atol=0)
    np.testing.assert_allclose(1.0 / F[:, 1], [4.0, 4.0, 2.75], rtol=0, atol=1e-15)
    np.testing.assert_allclose([F[0, 2], F[1, 2]], [2.0, 1.0], rtol=0, atol=0)


@pytest.mark.parametrize("n,b", [(1, 0), (6, 1), (40, 5), (130, 20), (97, 96)])
def test_reconstructs_and_matches_partial_pivoting(n, b):
    A = column_dominant_band(n, b, seed=n + b)
    F = B.lu_nopivot(B.dense_to_band(A, b))
    L, U = B.factors_dense(F)
    np.testing.assert_allclose(L @ U, A, rtol=0, atol=1e-12 * np.abs(A).max())
    P, Ls, Us = sla.lu(A)
    np.testing.assert_array_equal(P, np.eye(n))
    np.testing.assert_allclose(L, Ls, rtol=0, atol=1e-13)
    np.testing.assert_allclose(U, Us, rtol=0, atol=1e-12 * np.abs(A).max())
    # no fill outside the band
    assert np.all(np.abs(np.tril(L, -b - 1)) == 0) and np.all(np.abs(np.triu(U, b + 1)) == 0)


def test_zero_pivot_is_reported():
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(ZeroDivisionError):
        B.lu_nopivot(B.dense_to_band(A, 1))
