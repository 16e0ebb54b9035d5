"""The coarse factorization of Eq. 9 (A_0 = P_0^T DF P_0, no pivoting) through the C ABI
(nls_band_solve), against FP64 references on the CPU.

* Factors, backward error, entry by entry: |A - L U| <= 4 (b + 1) u |L| |U| (the textbook bound
  for Gaussian elimination, Higham, Accuracy and Stability of Numerical Algorithms, Thm. 9.3, with
  at most b + 1 terms per entry), u = 2^-53 for FP64 factors, and for FP32 factors 2^-21: the
  trailing products on the tensor cores use TF32 hi/lo splits, whose dropped lo*lo term and TF32
  reading of the lo parts are about 2^-22 of each product.
* Factors, forward, entry by entry, against the oracle's band LU without pivoting
  (oracle/banded.py), on the diagonally dominant matrices (growth below 2, a well-conditioned
  elimination): FP64 factors to 1e-12 of the largest factor entry, FP32 factors to 2e-5 of it
  (a few FP32 roundings).  The coarse matrices of the mechanics problems are checked through the
  backward error and the solve only: their elimination is ill-conditioned, so a forward bound
  would have to carry the condition number of the factorization.
* Solves, entry by entry, against a dense FP64 solve, to 10 kappa_inf(A) times the solve's
  residual target: FP64 factors 1e-15; FP32 factors refined in FP64 until ||g - A x|| <=
  1e-10 ||g||.
Matrices: column-diagonally-dominant random band matrices of ragged sizes (several tiles, a
partial last tile, half bandwidths below, at and above one tile), the coarse matrix of a 64 x 64
Neo-Hooke problem with 16 x 16 uneven subdomains, and a leading block and the whole of the
2048 x 2048 Neo-Hooke workload's coarse matrix (23,376 coarse dofs, half bandwidth 389).
"""
import numpy as np
import pytest

from oracle import banded as B
from paper_2410_24138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


def column_dominant_band(n, b, seed):
    rng = np.random.default_rng(seed)
    band = np.zeros((n, 2 * b + 1))
    for i in range(n):
        lo, hi = max(0, i - b), min(n, i + b + 1)
        band[i, lo - i + b:hi - i + b] = rng.uniform(-1.0, 1.0, hi - lo)
    A = B.band_to_dense(band)
    for j in range(n):
        A[j, j] = np.sign(A[j, j] or 1.0) * (np.abs(A[:, j]).sum() + 0.5)
    return B.dense_to_band(A, b)


def check(nls, band, precision, method, seed=0, forward_factors=True):
    n, w = band.shape
    b = (w - 1) // 2
    g = np.random.default_rng(seed).uniform(-1.0, 1.0, n)
    x, F = nls.band_solve(band, g, precision=precision, method=method, want_factors=True)
    A = B.band_to_dense(band)
    f64 = precision == nls.PREC_FP64
    # backward error of the factors
    L, U = B.factors_dense(F)
    u = 2.0 ** -53 if f64 else 2.0 ** -21
    bound = 4 * (b + 1) * u * (np.abs(L) @ np.abs(U))
    assert np.all(np.abs(A - L @ U) <= bound + 1e-300), (np.abs(A - L @ U) / (bound + 1e-300)).max()
    # forward error of the factors against the oracle's elimination
    if forward_factors:
        Fo = B.lu_nopivot(band)
        ftol = (1e-12 if f64 else 2e-5) * np.abs(Fo).max()
        assert np.abs(F - Fo).max() <= ftol, np.abs(F - Fo).max() / np.abs(Fo).max()
    # the solve
    xs = np.linalg.solve(A, g)
    kappa = np.linalg.cond(A, np.inf)
    xtol = 10 * kappa * (1e-15 if f64 else 1e-10) * np.abs(xs).max()
    assert np.abs(x - xs).max() <= xtol, (np.abs(x - xs).max() / np.abs(xs).max(), kappa)
    return x


@pytest.mark.parametrize("n,b", [(1, 0), (100, 3), (128, 64), (300, 127), (517, 129), (1000, 389), (777, 200)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tiles_match_the_oracle_lu_and_a_dense_solve(nls, n, b, precision):
    prec = nls.PREC_FP32_IR if precision == "fp32" else nls.PREC_FP64
    check(nls, column_dominant_band(n, b, seed=n * 7 + b), prec, nls.COARSE_FACTOR_TILES)


@pytest.mark.parametrize("n,b", [(100, 3), (300, 90)])
def test_one_cta_band_lu_matches_the_same_references(nls, n, b):
    for prec in (nls.PREC_FP32_IR, nls.PREC_FP64):
        check(nls, column_dominant_band(n, b, seed=n + b), prec, nls.COARSE_FACTOR_BAND)


def test_band_solve_refuses_what_it_cannot_factor(nls):
    with pytest.raises(nls.NLSError) as err:
        nls.band_solve(column_dominant_band(600, 200, 1), np.ones(600), method=nls.COARSE_FACTOR_BAND)
    assert err.value.status == -4  # NLS_E_UNSUPPORTED: half bandwidth above the one-CTA LU's 128
    with pytest.raises(nls.NLSError) as err:  # an FP64 window of 137 rows x 255 values exceeds shared memory
        nls.band_solve(column_dominant_band(300, 127, 1), np.ones(300), precision=nls.PREC_FP64,
                       method=nls.COARSE_FACTOR_BAND)
    assert err.value.status == -4
    band = np.zeros((3, 3))
    band[:, 1] = [1.0, 0.0, 1.0]
    with pytest.raises(nls.NLSError) as err:
        nls.band_solve(band, np.ones(3), method=nls.COARSE_FACTOR_TILES)
    assert err.value.status == -6  # NLS_E_PIVOT


@pytest.fixture(scope="module")
def neohooke_a0(nls):
    """A_0 = P_0^T DF(u_0) P_0 of a 64 x 64 Neo-Hooke problem (16 x 16 uneven subdomains) at a
    bending state, as the hybrid F_x evaluation forms it."""
    n = 64
    p = I.neohooke_problem(n, I.brick_partition(n, 16, 16, 5), 256, 2, 8.0)
    s = nls.make_solver(p, coupling="hybrid", precision="fp64")
    u = np.zeros(p.n_nodes * 2)
    u[1::2] = -0.02 * p.xy[:, 0] ** 2
    s.eval_Fx(u, 0.2)
    A0 = s.coarse_matrix()
    s.close()
    return A0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("method", ["tiles", "band"])
def test_neohooke_64_coarse_matrix(nls, neohooke_a0, precision, method):
    prec = nls.PREC_FP32_IR if precision == "fp32" else nls.PREC_FP64
    meth = nls.COARSE_FACTOR_TILES if method == "tiles" else nls.COARSE_FACTOR_BAND
    assert neohooke_a0.shape[0] > 256  # several tiles
    if method == "band" and (neohooke_a0.shape[1] - 1) // 2 > (128 if precision == "fp32" else 100):
        pytest.skip("half bandwidth beyond the one-CTA LU's shared-memory window")
    check(nls, neohooke_a0, prec, meth, seed=3, forward_factors=False)


@pytest.fixture(scope="module")
def c5_a0(nls):
    """A_0 of the 2048 x 2048 Neo-Hooke workload (23,376 coarse dofs, half bandwidth 389) as the
    hybrid F_x evaluation forms it in the chosen form (FP32 tiled coarse factorization), at the
    first load step's traction and a smooth bending state; the evaluation itself must succeed."""
    p = I.neohooke_c5()
    s = nls.make_solver(p, coupling="hybrid", precision="fp32", autotune=1)
    u = np.zeros(p.n_nodes * 2)
    u[1::2] = -0.02 * p.xy[:, 0] ** 2
    Fx, its, st = s.eval_Fx(u, 0.2)
    assert np.all(st == 0) and np.all(np.isfinite(Fx))
    A0 = s.coarse_matrix()
    s.close()
    return A0


def test_c5_coarse_matrix_leading_block(nls, c5_a0):
    """A leading principal block of C5's A_0 (2,048 rows: 16 tiles, 4 tile diagonals each side),
    factored and solved in both precisions against the oracle's LU and a dense FP64 solve."""
    n0, w = c5_a0.shape
    b = (w - 1) // 2
    assert n0 == 23376 and b == 389
    m = 2048
    sub = c5_a0[:m].copy()
    for i in range(m):
        hi = m - i + b  # columns >= m fall outside the block
        if hi < w:
            sub[i, hi:] = 0.0
    for prec in (nls.PREC_FP32_IR, nls.PREC_FP64):
        check(nls, sub, prec, nls.COARSE_FACTOR_TILES, seed=9, forward_factors=False)


def test_c5_coarse_matrix_whole(nls, c5_a0):
    """The whole of C5's A_0: the refined FP32 solve meets its stopping test in FP64 on the host
    (||g - A_0 x|| <= 1e-10 ||g||, a property at any size), and agrees with the FP64 tiled solve
    and with a sparse direct FP64 solve to within the condition number times that residual."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n0, w = c5_a0.shape
    b = (w - 1) // 2
    rows = np.repeat(np.arange(n0), w)
    cols = rows - b + np.tile(np.arange(w), n0)
    ok = (cols >= 0) & (cols < n0)
    A = sp.csr_matrix((c5_a0.ravel()[ok], (rows[ok], cols[ok])), shape=(n0, n0))
    g = np.random.default_rng(4).uniform(-1.0, 1.0, n0)
    x32 = nls.band_solve(c5_a0, g, precision=nls.PREC_FP32_IR, method=nls.COARSE_FACTOR_TILES)
    x64 = nls.band_solve(c5_a0, g, precision=nls.PREC_FP64, method=nls.COARSE_FACTOR_TILES)
    lu = spla.splu(A.tocsc())
    xs = lu.solve(g)
    r32 = np.linalg.norm(g - A @ x32) / np.linalg.norm(g)
    r64 = np.linalg.norm(g - A @ x64) / np.linalg.norm(g)
    rs = np.linalg.norm(g - A @ xs) / np.linalg.norm(g)
    assert r32 <= 2e-10, r32
    assert r64 <= 1e3 * max(rs, 1e-16), (r64, rs)
    # ||x - xs|| / ||xs|| <= kappa (||r|| + ||r_s||) / ||g||, kappa from a 1-norm estimate of A^-1
    inv = spla.LinearOperator((n0, n0), matvec=lu.solve, rmatvec=lambda v: lu.solve(v, trans="T"))
    kappa = spla.onenormest(A) * spla.onenormest(inv)
    for x, r in ((x32, r32), (x64, r64)):
        err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        assert err <= 100 * kappa * (r + rs), (err, kappa, r)
