// Device building blocks of the nonlinear Schwarz solver (sm_103a).
//
// * element routines of Eq. 1 (P1 nonlinear diffusion) and Eq. 2 (Q1 compressible Neo-Hooke),
// * block reductions with a fixed summation order (results do not depend on scheduling),
// * the no-pivoting band LU with a sliding shared-memory window over (b + 2) rows, reading
//   the assembled CSR rows of a local Jacobian and streaming finished factor rows to global
//   memory,
// * blocked forward / backward substitution with the band factors (one warp solves each
//   32-row diagonal block, the whole CTA applies its coupling to the next b rows).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nls_internal.h"

namespace nls {
namespace dev {

constexpr int kWarp = 32;

// ------------------------------------------------------------------------------------------
// reductions (deterministic for a fixed block size)
// ------------------------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread receives the result.  `red` holds >= 33 doubles.
__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------------------------------------------
// Eq. 1 on P1 triangles.  geo = {dphi_0/dx, dphi_0/dy, dphi_1/dx, ..., area, pad}.
// Residual of the element:  r_a = k Q (grad u . grad phi_a), Q = int_T (1 + u^2) by the
// exact edge-midpoint rule; the source term is handled through the external load vector.
// ------------------------------------------------------------------------------------------
struct P1State {
  double gx, gy, m01, m12, m20, kq, k, area;
};

__device__ inline P1State p1_state(const double* geo, double k, double u0, double u1, double u2) {
  P1State s;
  s.gx = u0 * geo[0] + u1 * geo[2] + u2 * geo[4];
  s.gy = u0 * geo[1] + u1 * geo[3] + u2 * geo[5];
  s.m01 = 0.5 * (u0 + u1);
  s.m12 = 0.5 * (u1 + u2);
  s.m20 = 0.5 * (u2 + u0);
  s.area = geo[6];
  s.k = k;
  const double Q = s.area * (1.0 / 3.0) * (3.0 + s.m01 * s.m01 + s.m12 * s.m12 + s.m20 * s.m20);
  s.kq = k * Q;
  return s;
}

__device__ inline void p1_residual(const double* geo, const P1State& s, double r[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = s.kq * (s.gx * geo[2 * a] + s.gy * geo[2 * a + 1]);
}

// K[a][b] = d r_a / d u_b = k Q grad phi_a . grad phi_b + k (grad u . grad phi_a) dQ/du_b
template <typename T>
__device__ inline void p1_jacobian(const double* geo, const P1State& s, T K[9]) {
  const double a3 = s.area * (1.0 / 3.0);
  const double dQ[3] = {a3 * (s.m01 + s.m20), a3 * (s.m01 + s.m12), a3 * (s.m12 + s.m20)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double flux = s.gx * geo[2 * a] + s.gy * geo[2 * a + 1];
#pragma unroll
    for (int b = 0; b < 3; ++b)
      K[a * 3 + b] = (T)(s.kq * (geo[2 * a] * geo[2 * b] + geo[2 * a + 1] * geo[2 * b + 1]) + s.k * flux * dQ[b]);
  }
}

// ------------------------------------------------------------------------------------------
// Eq. 2 on Q1 quadrilaterals, 2x2 Gauss.  geo per Gauss point q (stride 10): dN_a/dX (4 x 2)
// then weight * det(dX/dxi).  P = mu F - (mu - lambda ln J) F^-T.
// With p_a = F^-1 applied from the left to grad N_a (p_a[i] = sum_J gradN_a[J] Finv[J][i]):
//   r_{a,i}      = w [ mu (F gradN_a)_i - (mu - lambda ln J) p_a[i] ]
//   K_{ai, bk}   = w [ mu delta_ik gradN_a . gradN_b + lambda p_a[i] p_b[k] + (mu - lambda ln J) p_a[k] p_b[i] ]
// ------------------------------------------------------------------------------------------
template <typename T>
struct NHPoint {
  T F00, F01, F10, F11, i00, i01, i10, i11, c, w;  // c = mu - lambda ln J
  bool ok;
};

template <typename T>
__device__ inline NHPoint<T> nh_point(const double* g, const T u[8], T mu, T lam) {
  NHPoint<T> p;
  p.F00 = 1;
  p.F01 = 0;
  p.F10 = 0;
  p.F11 = 1;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const T bx = (T)g[2 * a], by = (T)g[2 * a + 1];
    p.F00 += u[2 * a] * bx;
    p.F01 += u[2 * a] * by;
    p.F10 += u[2 * a + 1] * bx;
    p.F11 += u[2 * a + 1] * by;
  }
  const T det = p.F00 * p.F11 - p.F01 * p.F10;
  p.ok = det > (T)0;
  const T inv = (T)1 / det;
  p.i00 = p.F11 * inv;
  p.i01 = -p.F01 * inv;
  p.i10 = -p.F10 * inv;
  p.i11 = p.F00 * inv;
  p.c = mu - lam * (p.ok ? log(det) : (T)0);
  p.w = (T)g[8];
  return p;
}

__device__ inline void nh_residual(const double* geo, const double u[8], double mu, double lam, double r[8], bool& ok) {
#pragma unroll
  for (int k = 0; k < 8; ++k) r[k] = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double* g = geo + q * 10;
    NHPoint<double> p = nh_point<double>(g, u, mu, lam);
    ok = ok && p.ok;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double bx = g[2 * a], by = g[2 * a + 1];
      const double pa0 = bx * p.i00 + by * p.i10, pa1 = bx * p.i01 + by * p.i11;
      r[2 * a] += p.w * (mu * (p.F00 * bx + p.F01 * by) - p.c * pa0);
      r[2 * a + 1] += p.w * (mu * (p.F10 * bx + p.F11 * by) - p.c * pa1);
    }
  }
}

template <typename T>
__device__ inline void nh_jacobian(const double* geo, const double ud[8], double mud, double lamd, T K[64]) {
  T u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) u[k] = (T)ud[k];
  const T mu = (T)mud, lam = (T)lamd;
#pragma unroll
  for (int k = 0; k < 64; ++k) K[k] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double* g = geo + q * 10;
    NHPoint<T> p = nh_point<T>(g, u, mu, lam);
    T bx[4], by[4], p0[4], p1[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      bx[a] = (T)g[2 * a];
      by[a] = (T)g[2 * a + 1];
      p0[a] = bx[a] * p.i00 + by[a] * p.i10;
      p1[a] = bx[a] * p.i01 + by[a] * p.i11;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const T gg = mu * (bx[a] * bx[b] + by[a] * by[b]);
        // rows (a, i), cols (b, k)
        K[(2 * a + 0) * 8 + 2 * b + 0] += p.w * (gg + lam * p0[a] * p0[b] + p.c * p0[a] * p0[b]);
        K[(2 * a + 0) * 8 + 2 * b + 1] += p.w * (lam * p0[a] * p1[b] + p.c * p1[a] * p0[b]);
        K[(2 * a + 1) * 8 + 2 * b + 0] += p.w * (lam * p1[a] * p0[b] + p.c * p0[a] * p1[b]);
        K[(2 * a + 1) * 8 + 2 * b + 1] += p.w * (gg + lam * p1[a] * p1[b] + p.c * p1[a] * p1[b]);
      }
  }
}

// The Gauss-point state of Eq. 2 that the tangent needs (c = mu - lambda ln J, weight, F^-1),
// computed once per element; nh_tangent_rows then forms the two rows of one node at a time, so
// that the 64 FP64 entries of the element tangent are never live at once.
struct NHGauss {
  double c[4], w[4], i00[4], i01[4], i10[4], i11[4];
};

__device__ inline void nh_gauss(const double* geo, const double u[8], double mu, double lam, NHGauss& G) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const NHPoint<double> p = nh_point<double>(geo + q * 10, u, mu, lam);
    G.c[q] = p.c;
    G.w[q] = p.w;
    G.i00[q] = p.i00;
    G.i01[q] = p.i01;
    G.i10[q] = p.i10;
    G.i11[q] = p.i11;
  }
}

// Rows (a, 0) and (a, 1) of the element tangent K of Eq. 2 (the same entries as nh_jacobian):
// R[i * 8 + 2 b + k] = K_{(a,i),(b,k)}.
__device__ inline void nh_tangent_rows(const double* geo, const NHGauss& G, double mu, double lam, int a, double R[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) R[k] = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double* g = geo + q * 10;
    const double bxa = g[2 * a], bya = g[2 * a + 1];
    const double p0a = bxa * G.i00[q] + bya * G.i10[q], p1a = bxa * G.i01[q] + bya * G.i11[q];
    const double w = G.w[q], c = G.c[q];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const double bx = g[2 * b], by = g[2 * b + 1];
      const double p0b = bx * G.i00[q] + by * G.i10[q], p1b = bx * G.i01[q] + by * G.i11[q];
      const double gg = mu * (bxa * bx + bya * by);
      R[2 * b + 0] += w * (gg + lam * p0a * p0b + c * p0a * p0b);
      R[2 * b + 1] += w * (lam * p0a * p1b + c * p1a * p0b);
      R[8 + 2 * b + 0] += w * (lam * p1a * p0b + c * p0a * p1b);
      R[8 + 2 * b + 1] += w * (gg + lam * p1a * p1b + c * p1a * p1b);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Band LU without pivoting.  Rows of the matrix come from a CSR block (columns are table dof
// indices; only columns < n belong to the local matrix) or from a dense band array.
// Factor layout (row-major band, W = 2b + 1 entries per row): d < b holds L[i][i-b+d],
// d = b holds 1 / U[i][i], d > b holds U[i][i+d-b].
// ------------------------------------------------------------------------------------------
struct RowSource {
  const int32_t* rowptr;  // nullptr: dense band rows in `val` (W entries per row)
  const int32_t* colidx;
  const double* val;
};

template <typename FT>
__device__ inline void load_band_row_warp(int row, int n, int b, const RowSource& src, FT* dst) {
  const int W = 2 * b + 1, lane = threadIdx.x & 31;
  if (src.rowptr == nullptr) {
    for (int d = lane; d < W; d += 32) dst[d] = (row < n) ? (FT)src.val[(int64_t)row * W + d] : (FT)0;
    __syncwarp();
    return;
  }
  for (int d = lane; d < W; d += 32) dst[d] = (FT)0;
  __syncwarp();
  if (row < n) {
    const int k1 = src.rowptr[row + 1];
    for (int k = src.rowptr[row] + lane; k < k1; k += 32) {
      const int col = src.colidx[k];
      if (col < n) dst[col - row + b] = (FT)src.val[k];
    }
  }
  __syncwarp();
}

// Returns (to every thread) 0 on success, 1 if a pivot was zero or not finite.
// smem: win [(b + 2) * (2b + 1)], rp [b + 2], flag [1].
template <typename FT>
__device__ int band_lu(int n, int b, const RowSource& src, FT* __restrict__ F, FT* win, FT* rp, int* flag) {
  const int W = 2 * b + 1, R = b + 2;
  const int tid = threadIdx.x, T = blockDim.x, wid = tid >> 5, nw = T >> 5;
  if (n <= 0) return 0;
  if (tid == 0) *flag = 0;
  // rows 0..b into slots 0..b
  for (int i = wid; i <= b; i += nw) load_band_row_warp<FT>(i, n, b, src, win + (i % R) * W);
  __syncthreads();
  if (tid == 0) {
    const FT p = win[b];
    if (!(p != (FT)0) || !isfinite((double)p)) *flag = 1;
    rp[0] = (FT)1 / p;
  }
  __syncthreads();
  const int bb = b * b;
  const int dq = (b > 0) ? T / b : 0, dr = (b > 0) ? T % b : 0;
  const int ri0 = (b > 0) ? tid / b : 0, cj0 = (b > 0) ? tid % b : 0;
  for (int k = 0; k < n; ++k) {
    const int sk = k % R;
    const FT* rowk = win + sk * W;
    const FT rpk = rp[sk];
    const int lim = min(b, n - 1 - k);
    // warp 0: write back row k (scaled L part, reciprocal pivot) and stage row k + b + 1
    if (wid == 0) {
      FT* out = F + (int64_t)k * W;
      for (int d = tid; d < W; d += 32) {
        const int j = k - b + d;
        FT v = rowk[d];
        if (d < b) v = (j >= 0) ? v * rp[j % R] : (FT)0;
        else if (d == b) v = rpk;
        out[d] = v;
      }
      load_band_row_warp<FT>(k + b + 1, n, b, src, win + ((k + b + 1) % R) * W);
    }
    // rank-1 update of rows k+1..k+lim, columns k+1..k+lim
    if (lim > 0) {
      const int base = (k + 1) % R;
      int ri = ri0, cj = cj0;
      for (int idx = tid; idx < bb; idx += T) {
        if (ri < lim && cj < lim) {
          int slot = base + ri;
          if (slot >= R) slot -= R;
          FT* rowi = win + slot * W;
          const FT l = rowi[b - 1 - ri] * rpk;
          const FT nv = rowi[cj - ri + b] - l * rowk[b + 1 + cj];
          rowi[cj - ri + b] = nv;
          if (idx == 0) {
            if (!(nv != (FT)0) || !isfinite((double)nv)) *flag = 1;
            rp[(k + 1) % R] = (FT)1 / nv;
          }
        }
        cj += dr;
        ri += dq;
        if (cj >= b) {
          cj -= b;
          ri += 1;
        }
      }
    } else if (tid == 0 && k + 1 < n) {
      const FT nv = win[((k + 1) % R) * W + b];
      if (!(nv != (FT)0) || !isfinite((double)nv)) *flag = 1;
      rp[(k + 1) % R] = (FT)1 / nv;
    }
    __syncthreads();
  }
  return *flag;
}

// ------------------------------------------------------------------------------------------
// In-place band LU with asynchronous row staging.  F holds the assembled band rows on entry
// (row-major, W = 2b + 1) and the factors on exit (layout as above).  Rows are copied into the
// shared-memory ring with cp.async PD rows ahead of use, so the global-memory latency of a
// row overlaps the PD elimination steps before it is needed; each row is read exactly once
// and written back exactly once.
// smem: win [(b + 2 + PD) * W], rp [b + 2 + PD], flag [1].
// ------------------------------------------------------------------------------------------
template <typename FT>
__device__ inline void cp_async_elem(FT* sdst, const FT* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if (sizeof(FT) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One warp stages band row `row` (if it exists) into dst and commits one copy group per lane.
template <typename FT>
__device__ inline void stage_row_async(int row, int n, int W, const FT* F, FT* dst) {
  const int lane = threadIdx.x & 31;
  if (row < n) {
    const FT* src = F + (int64_t)row * W;
    for (int d = lane; d < W; d += 32) cp_async_elem<FT>(dst + d, src + d);
  }
  cp_async_commit();
}

constexpr int kLuPrefetch = 8;

// Rows of the shared-memory window of the band LU: the b + 2 rows an elimination step touches
// plus the rows staged ahead.
__host__ __device__ constexpr int band_lu_window_rows(int b) { return b + 2 + kLuPrefetch; }

// Row stride of the window (>= 2b + 1 entries).  One warp of the 2D-tiled update touches 4
// consecutive rows x 8 consecutive columns, at addresses (stride - 1) apart from row to row;
// with (stride - 1) = 8 or 24 (mod 32) the four rows land on disjoint groups of 8 banks.
__host__ __device__ constexpr int band_lu_window_stride(int b) {
  int w = 2 * b + 1;
  while (((w - 1) & 31) != 8 && ((w - 1) & 31) != 24) ++w;
  return w;
}

// Thread mapping of one elimination step (2D tiling): the CTA is TY x 8 threads, thread
// (ty, tx) updates rows k+1+ri with ri = ty, ty + TY, ... and columns k+1+cj with
// cj = tx, tx + 8, ..., tx + 8 (QM - 1) (b <= 8 QM).  Every thread loads its QM pivot-row
// values once per step and one multiplier per row, so the per-row overhead is shared by QM
// entries and at most 7 column slots per row are idle.  Every thread forms 1 / pivot itself
// after the step's barrier (no single-thread step on the critical path); thread 0 records it
// in rp (per ring slot) for the write-back of the L part and flags a bad pivot.
template <typename FT>
__device__ inline FT recip(FT p) {
  if constexpr (sizeof(FT) == 4) return __frcp_rn(p);
  else return (FT)1 / p;
}

template <typename FT, int QM>
__device__ int band_lu_inplace_q(int n, int b, FT* __restrict__ F, FT* win, FT* rp, int* flag) {
  constexpr int PD = kLuPrefetch, TX = 8;
  const int W = 2 * b + 1, WS = band_lu_window_stride(b), R = b + 2 + PD;
  const int tid = threadIdx.x, T = blockDim.x, tx = tid % TX, ty = tid / TX, TY = T / TX;
  if (tid == 0) *flag = 0;
  // stage rows 0 .. b + PD (one copy group per row and thread)
  for (int i = 0; i <= b + PD; ++i) {
    if (i < n)
      for (int d = tid; d < W; d += T) cp_async_elem<FT>(win + i * WS + d, F + (int64_t)i * W + d);
    cp_async_commit();
  }
  cp_async_wait<PD>();
  __syncthreads();
  int sk = 0, s1 = 1;  // ring slots of rows k and k + 1 (R >= b + 2 >= 2)
  for (int k = 0; k < n; ++k) {
    const FT* rowk = win + sk * WS;
    const FT piv = rowk[b];
    const FT rpk = recip<FT>(piv);
    if (tid == 0) {
      if (!(piv != (FT)0) || !isfinite((double)piv)) *flag = 1;
      rp[sk] = rpk;
    }
    const int lim = min(b, n - 1 - k);
    // row k is final: write it back in place (scaled L part, reciprocal pivot, U part)
    for (int d = tid; d < W; d += T) {
      FT v = rowk[d];
      if (d < b) {
        int sj = sk - b + d;
        if (sj < 0) sj += R;
        v = (k - b + d >= 0) ? v * rp[sj] : (FT)0;
      } else if (d == b) {
        v = rpk;
      }
      F[(int64_t)k * W + d] = v;
    }
    // stage row k + b + 1 + PD into the slot row k - 1 used
    {
      const int rs = k + b + 1 + PD;
      const int ss = (sk == 0) ? R - 1 : sk - 1;
      if (rs < n)
        for (int d = tid; d < W; d += T) cp_async_elem<FT>(win + ss * WS + d, F + (int64_t)rs * W + d);
      cp_async_commit();
    }
    // rank-1 update of rows k+1..k+lim, columns k+1..k+lim
    FT u[QM];
#pragma unroll
    for (int q = 0; q < QM; ++q) u[q] = (tx + TX * q < lim) ? rowk[b + 1 + tx + TX * q] : (FT)0;
    for (int ri = ty; ri < lim; ri += TY) {
      int slot = s1 + ri;
      if (slot >= R) slot -= R;
      FT* rowi = win + slot * WS + b - ri;
      const FT l = rowi[-1] * rpk;
#pragma unroll
      for (int q = 0; q < QM; ++q) {
        const int cj = tx + TX * q;
        if (cj < lim) rowi[cj] -= l * u[q];
      }
    }
    // rows up to k + b + 1 must have landed before step k + 1
    cp_async_wait<PD>();
    __syncthreads();
    sk = s1;
    s1 = (s1 + 1 == R) ? 0 : s1 + 1;
  }
  cp_async_wait<0>();
  __syncthreads();
  return *flag;
}


// Dispatch on the number of column slots per thread (half bandwidth up to 128).  blockDim.x
// must be a multiple of 8.
template <typename FT>
__device__ int band_lu_inplace(int n, int b, FT* __restrict__ F, FT* win, FT* rp, int* flag) {
  if (n <= 0) return 0;
  if (b <= 32) return band_lu_inplace_q<FT, 4>(n, b, F, win, rp, flag);
  if (b <= 48) return band_lu_inplace_q<FT, 6>(n, b, F, win, rp, flag);
  if (b <= 64) return band_lu_inplace_q<FT, 8>(n, b, F, win, rp, flag);
  if (b <= 96) return band_lu_inplace_q<FT, 12>(n, b, F, win, rp, flag);
  return band_lu_inplace_q<FT, 16>(n, b, F, win, rp, flag);
}

// ------------------------------------------------------------------------------------------
// Triangular solves with the band factors, in place on y[0..n) (shared memory).
// ------------------------------------------------------------------------------------------
// Block size of the triangular solves: 32 rows (one warp) for FP32 factors, 16 for FP64
// (two register sets of BS values per thread stay within the register budget).
template <typename FT>
struct SolveBlock {
  static constexpr int BS = sizeof(FT) == 4 ? 32 : 16;
};

// The factor values of block k0 + BS are loaded into registers while block k0 is solved, so
// the global-memory latency of the next block overlaps the current one.
//
// Roles: warp 0 solves the BS x BS diagonal block; threads 32 .. 32 + b - 1 each own one of the
// b rows coupled to the block.  Both roles keep their current and next values in the same two
// register arrays (Dcur/Dnxt), so a thread holds 2 BS values.  Needs blockDim.x >= 32 + b.
template <typename FT>
__device__ void band_solve(int n, int b, const FT* __restrict__ F, FT* y) {
  constexpr int BS = SolveBlock<FT>::BS;
  const int W = 2 * b + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool diag = wid == 0;
  const bool offd = tid >= 32 && tid < 32 + b;
  const int r = tid - 32;
  FT cur[BS], nxt[BS];
  // forward (unit lower L): block k0 = rows [k0, k0 + kb)
#define NLS_LOAD_FWD(k0_, R_)                                                             \
  {                                                                                       \
    const int kb_ = min(BS, n - (k0_));                                                   \
    if (diag) {                                                                           \
      _Pragma("unroll") for (int j = 0; j < BS; ++j) {                                    \
        const int d = j - lane + b;                                                       \
        R_[j] = (j < lane && lane < kb_ && d >= 0) ? F[(int64_t)((k0_) + lane) * W + d] : (FT)0; \
      }                                                                                   \
    } else if (offd) {                                                                    \
      const int i_ = (k0_) + kb_ + r;                                                     \
      _Pragma("unroll") for (int j = 0; j < BS; ++j) {                                    \
        const int d = j + b - kb_ - r;                                                    \
        R_[j] = (i_ < n && j < kb_ && d >= 0) ? F[(int64_t)i_ * W + d] : (FT)0;           \
      }                                                                                   \
    }                                                                                     \
  }
  if (n > 0) NLS_LOAD_FWD(0, cur);
  for (int k0 = 0; k0 < n; k0 += BS) {
    const int kb = min(BS, n - k0);
    if (k0 + BS < n) NLS_LOAD_FWD(k0 + BS, nxt);
    if (diag) {
      FT yl = (lane < kb) ? y[k0 + lane] : (FT)0;
#pragma unroll
      for (int j = 0; j < BS; ++j) {
        const FT yj = __shfl_sync(0xffffffffu, yl, j);
        if (j < kb) yl -= cur[j] * yj;
      }
      if (lane < kb) y[k0 + lane] = yl;
    }
    __syncthreads();
    if (offd) {
      const int i = k0 + kb + r;
      if (i < n) {
        FT acc = 0;
#pragma unroll
        for (int j = 0; j < BS; ++j)
          if (j < kb) acc += cur[j] * y[k0 + j];
        y[i] -= acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < BS; ++j) cur[j] = nxt[j];
  }
#undef NLS_LOAD_FWD
  // backward (U, diagonal stored inverted): block rows [k0, k1)
#define NLS_LOAD_BWD(k1_, R_)                                                             \
  {                                                                                       \
    const int k0_ = max(0, (k1_) - BS), kb_ = (k1_) - k0_;                                \
    if (diag) {                                                                           \
      _Pragma("unroll") for (int j = 0; j < BS; ++j) {                                    \
        const int d = j - lane + b;                                                       \
        R_[j] = (j >= lane && lane < kb_ && j < kb_ && d <= 2 * b) ? F[(int64_t)(k0_ + lane) * W + d] : (FT)0; \
      }                                                                                   \
    } else if (offd) {                                                                    \
      const int i_ = k0_ - 1 - r;                                                         \
      _Pragma("unroll") for (int j = 0; j < BS; ++j) {                                    \
        R_[j] = (i_ >= 0 && j < kb_ && j + 1 + r <= b) ? F[(int64_t)i_ * W + (j + 1 + r + b)] : (FT)0; \
      }                                                                                   \
    }                                                                                     \
  }
  if (n > 0) NLS_LOAD_BWD(n, cur);
  for (int k1 = n; k1 > 0; k1 -= BS) {
    const int k0 = max(0, k1 - BS), kb = k1 - k0;
    if (k0 > 0) NLS_LOAD_BWD(k0, nxt);
    if (diag) {
      FT yl = (lane < kb) ? y[k0 + lane] : (FT)0;
#pragma unroll
      for (int j = BS - 1; j >= 0; --j) {
        if (j < kb) {
          FT xj = (lane == j) ? yl * cur[j] : (FT)0;
          xj = __shfl_sync(0xffffffffu, xj, j);
          if (lane == j) yl = xj;
          else if (lane < j) yl -= cur[j] * xj;
        }
      }
      if (lane < kb) y[k0 + lane] = yl;
    }
    __syncthreads();
    if (offd) {
      const int i = k0 - 1 - r;
      if (i >= 0) {
        FT acc = 0;
#pragma unroll
        for (int j = 0; j < BS; ++j)
          if (j < kb) acc += cur[j] * y[k0 + j];
        y[i] -= acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < BS; ++j) cur[j] = nxt[j];
  }
#undef NLS_LOAD_BWD
}

// ------------------------------------------------------------------------------------------
// Packed solve operands.  After a factorization the operands of the two triangular solves are
// copied, block by block (BS rows), into a layout in which every warp-wide load of the solve
// reads BS consecutive values:
//
//   block t (rows k0 = t BS .. k0 + bs - 1), PB = 2 BS^2 + 2 b BS entries:
//     [0, BS^2)               inv(L_tt), column-major: entry (r, j) at j BS + r (identity padded)
//     [BS^2, 2 BS^2)          inv(U_tt), column-major (U's diagonal is stored inverted)
//     [2 BS^2, + b BS)        CL: entry (j, r) at j b + r = L[k0 + BS + r][k0 + j]
//     [2 BS^2 + b BS, + b BS) CU: entry (j, r) at j b + r = U[k0 - 1 - r][k0 + j]
//
// The explicit diagonal-block inverses replace the BS-step dependent shuffle chain of a
// diagonal block by one short dot product per row.  One warp per block; `tmp` holds
// BS x (BS + 1) FT per warp that takes part (`nwarps`).
// ------------------------------------------------------------------------------------------
template <typename FT>
__host__ __device__ constexpr int64_t packed_block_entries(int b) {
  return 2 * (int64_t)SolveBlock<FT>::BS * SolveBlock<FT>::BS + 2 * (int64_t)b * SolveBlock<FT>::BS;
}

// Blocks t = first + wid, first + wid + stride, ... are packed by warp `wid` (< nwarps); one CTA
// packing everything passes first = 0, stride = nwarps, several CTAs pass their own offsets.
template <typename FT>
__device__ void band_pack_solve_range(int n, int b, const FT* __restrict__ F, FT* __restrict__ P, FT* tmp, int nwarps,
                                      int first, int stride) {
  constexpr int BS = SolveBlock<FT>::BS;
  const int W = 2 * b + 1, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = (n + BS - 1) / BS;
  const int64_t PB = packed_block_entries<FT>(b);
  if (wid < nwarps) {
    FT* M = tmp + wid * BS * (BS + 1);
    for (int t = first + wid; t < nblk; t += stride) {
      const int k0 = t * BS, bs = min(BS, n - k0);
      FT* out = P + (int64_t)t * PB;
      // lower: M[i][j] = L[k0+i][k0+j] (j < i), unit diagonal
      for (int e = lane; e < BS * BS; e += 32) {
        const int i = e / BS, j = e % BS;
        FT v = (FT)0;
        if (i < bs && j < i && i - j <= b) v = F[(int64_t)(k0 + i) * W + (j - i + b)];
        M[i * (BS + 1) + j] = v;
      }
      __syncwarp();
      if (lane < BS) {
        // column `lane` of inv(L): forward substitution with e_lane
        FT x[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
          FT acc = (i == lane) ? (FT)1 : (FT)0;
#pragma unroll
          for (int j = 0; j < i; ++j) acc -= M[i * (BS + 1) + j] * x[j];
          x[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) out[lane * BS + i] = x[i];
      }
      __syncwarp();
      // upper: M[i][j] = U[k0+i][k0+j] (j > i), M[i][i] = 1/U_ii (stored reciprocal)
      for (int e = lane; e < BS * BS; e += 32) {
        const int i = e / BS, j = e % BS;
        FT v = (i == j) ? (FT)1 : (FT)0;
        if (i < bs && j < bs && j >= i && j - i <= b) v = F[(int64_t)(k0 + i) * W + (j - i + b)];
        M[i * (BS + 1) + j] = v;
      }
      __syncwarp();
      if (lane < BS) {
        // column `lane` of inv(U): backward substitution with e_lane (diagonal given inverted)
        FT x[BS];
#pragma unroll
        for (int i = BS - 1; i >= 0; --i) {
          FT acc = (i == lane) ? (FT)1 : (FT)0;
#pragma unroll
          for (int j = i + 1; j < BS; ++j) acc -= M[i * (BS + 1) + j] * x[j];
          x[i] = acc * M[i * (BS + 1) + i];
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) out[BS * BS + lane * BS + i] = x[i];
      }
      // couplings (coalesced writes; the band is read once per factorization)
      FT* cl = out + 2 * BS * BS;
      FT* cu = cl + (int64_t)b * BS;
      for (int e = lane; e < BS * b; e += 32) {
        const int j = e / b, r = e % b;
        const int il = k0 + BS + r, dl = j - BS - r + b;
        cl[e] = (j < bs && il < n && dl >= 0) ? F[(int64_t)il * W + dl] : (FT)0;
        const int iu = k0 - 1 - r;
        cu[e] = (j < bs && iu >= 0 && j + 1 + r <= b) ? F[(int64_t)iu * W + (j + 1 + r + b)] : (FT)0;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

template <typename FT>
__device__ void band_pack_solve(int n, int b, const FT* __restrict__ F, FT* __restrict__ P, FT* tmp, int nwarps) {
  band_pack_solve_range<FT>(n, b, F, P, tmp, nwarps, 0, nwarps);
}

// Triangular solves with the packed operands, in place on y[0..n) (shared memory): warp 0
// applies the block inverse (lane r: row r of inv(L_tt) or inv(U_tt) dotted with the block of
// y), threads 32 .. 32 + b - 1 apply the coupling to the next b rows.  With PF the operands of
// the next block are loaded into registers while the current one is applied (2 BS operand
// registers per thread: for kernels with few CTAs per SM, where nothing else hides the load
// latency); without PF each block's operands are loaded at the top of its step (BS registers,
// for kernels that keep enough CTAs resident).  With l2d > 0 the operands of the block l2d steps
// ahead are prefetched into L2 (one 128-byte line per thread: the diagonal-block inverse by the
// first BS^2 sizeof(FT) / 128 threads, the b coupling lines by the coupling threads), so that
// the register loads of the current and next block wait for L2 rather than HBM.  The forward
// sweep starts at block t0: y must vanish in the rows before it.  Needs blockDim.x >= 32 + b.
template <typename FT, bool PF>
__device__ void band_solve_packed(int n, int b, const FT* __restrict__ P, FT* y, int l2d = 0, int t0 = 0) {
  constexpr int BS = SolveBlock<FT>::BS;
  constexpr int NB = PF ? 2 : 1;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool diag = wid == 0 && lane < BS;
  const bool offd = tid >= 32 && tid < 32 + b;
  const int r = tid - 32;
  const int64_t PB = packed_block_entries<FT>(b);
  const int nblk = (n + BS - 1) / BS;
  const int64_t oL = 0, oU = BS * BS, oCL = 2 * BS * BS, oCU = 2 * BS * BS + (int64_t)b * BS;
  FT buf[NB][BS];
  auto load = [&](int t, int which, int64_t od, int64_t oc) {
    const FT* Pt = P + (int64_t)t * PB;
    if (diag) {
#pragma unroll
      for (int j = 0; j < BS; ++j) buf[which][j] = Pt[od + j * BS + lane];
    } else if (offd) {
#pragma unroll
      for (int j = 0; j < BS; ++j) buf[which][j] = Pt[oc + j * b + r];
    }
  };
  constexpr int LINE = 128 / (int)sizeof(FT);            // entries per 128-byte line
  constexpr int DLINES = BS * BS * (int)sizeof(FT) / 128;  // lines of one diagonal-block inverse
  auto l2pf = [&](int t, int64_t od, int64_t oc) {
    const FT* Pt = P + (int64_t)t * PB;
    const FT* a = nullptr;
    if (tid < DLINES) a = Pt + od + (int64_t)tid * LINE;
    else if (offd) a = Pt + oc + (int64_t)r * LINE;
    if (a) asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a)));
  };
  // forward: diag lanes read inv(L_tt), coupling threads read CL
  if (PF && t0 < nblk) load(t0, 0, oL, oCL);
  for (int q = t0 + 1; q < t0 + l2d && q < nblk; ++q) l2pf(q, oL, oCL);
  for (int t = t0; t < nblk; ++t) {
    const int k0 = t * BS, kb = min(BS, n - k0);
    if (l2d > 0 && t + l2d < nblk) l2pf(t + l2d, oL, oCL);
    if (PF) {
      if (t + 1 < nblk) load(t + 1, NB - 1, oL, oCL);
    } else {
      load(t, 0, oL, oCL);
    }
    const FT* cur = buf[0];
    if (wid == 0) {  // the whole warp reaches __syncwarp; only lanes < BS hold a block row
      FT a0 = 0, a1 = 0;
      if (diag) {
#pragma unroll
        for (int j = 0; j < BS; j += 2) {
          a0 += cur[j] * ((j < kb) ? y[k0 + j] : (FT)0);
          a1 += cur[j + 1] * ((j + 1 < kb) ? y[k0 + j + 1] : (FT)0);
        }
      }
      __syncwarp();
      if (lane < kb) y[k0 + lane] = a0 + a1;
    }
    __syncthreads();
    if (offd) {
      const int i = k0 + BS + r;
      if (i < n) {
        FT a0 = 0, a1 = 0;
#pragma unroll
        for (int j = 0; j < BS; j += 2) {
          a0 += cur[j] * y[k0 + j];
          a1 += cur[j + 1] * y[k0 + j + 1];
        }
        y[i] -= a0 + a1;
      }
    }
    __syncthreads();
    if (PF) {
#pragma unroll
      for (int j = 0; j < BS; ++j) buf[0][j] = buf[NB - 1][j];
    }
  }
  // backward: diag lanes read inv(U_tt), coupling threads read CU
  if (PF && nblk > 0) load(nblk - 1, 0, oU, oCU);
  for (int q = 1; q < l2d && nblk - 1 - q >= 0; ++q) l2pf(nblk - 1 - q, oU, oCU);
  for (int t = nblk - 1; t >= 0; --t) {
    const int k0 = t * BS, kb = min(BS, n - k0);
    if (l2d > 0 && t - l2d >= 0) l2pf(t - l2d, oU, oCU);
    if (PF) {
      if (t > 0) load(t - 1, NB - 1, oU, oCU);
    } else {
      load(t, 0, oU, oCU);
    }
    const FT* cur = buf[0];
    if (wid == 0) {
      FT a0 = 0, a1 = 0;
      if (diag) {
#pragma unroll
        for (int j = 0; j < BS; j += 2) {
          a0 += cur[j] * ((j < kb) ? y[k0 + j] : (FT)0);
          a1 += cur[j + 1] * ((j + 1 < kb) ? y[k0 + j + 1] : (FT)0);
        }
      }
      __syncwarp();
      if (lane < kb) y[k0 + lane] = a0 + a1;
    }
    __syncthreads();
    if (offd) {
      const int i = k0 - 1 - r;
      if (i >= 0) {
        FT a0 = 0, a1 = 0;
#pragma unroll
        for (int j = 0; j < BS; j += 2) {
          if (j < kb) a0 += cur[j] * y[k0 + j];
          if (j + 1 < kb) a1 += cur[j + 1] * y[k0 + j + 1];
        }
        y[i] -= a0 + a1;
      }
    }
    __syncthreads();
    if (PF) {
#pragma unroll
      for (int j = 0; j < BS; ++j) buf[0][j] = buf[NB - 1][j];
    }
  }
}

}  // namespace dev
}  // namespace nls
