// Device solver of the two-level nonlinear Schwarz method (sm_103a).
//
// Kernels:
//   k_local_newton   one persistent launch per F_x evaluation: every overlapping subdomain
//                    (longest first, pulled from a device work counter) runs its local
//                    Newton loop for Eq. 4 -- colour-ordered element assembly of the FP64
//                    residual and of the local Jacobian (CSR), sliding-window band LU in
//                    FP32 or FP64, triangular solves with FP64 iterative refinement, Armijo
//                    line search -- and refactors the Jacobian at the converged state for the
//                    exact tangent (Eq. 6 / Eq. 12).  It writes P~_i T_i straight into F_x.
//   k_local_apply    one CTA per subdomain: sum_i P~_i (R_i DF(v_i) P_i)^-1 R_i DF(v_i) y.
//   k_harmonic       energy-minimising extension of the RGDSW interface values (setup).
//   k_galerkin       per non-overlapping subdomain: Phi_j^T K^(j)(x) Phi_j (coarse matrix).
//   k_coarse_*       band LU / solve of A_0 = P_0^T DF P_0 in one CTA (Eq. 9).
//   k_elem_residual, k_node_residual   global residual F(u): element contributions, then fixed-order
//                    sums per node.
//   k_global_jacobian  colour-ordered global Jacobian DF(u) (Eq. 3).
//   k_vec_*          GMRES vector kernels with fixed-order (deterministic) reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <mutex>
#include <vector>

#include "dev_state.cuh"
#include "device.cuh"
#include "nls_internal.h"

namespace nls {

// coarse_tlu.cu
void tlu_prepare(Context& c, bool f32);
void tlu_factor(Context& c);
void tlu_free(Context& c);
bool tlu_solve(Context& c, const double* rhs, double* z, int accumulate, const int* skip, int* reset);
void tlu_check_solves(Context& c);

namespace {



constexpr int kVecBlocks = 1216;  // 8 per SM on 152 SMs
constexpr int kVecThreads = 256;
constexpr int kVecWarps = kVecBlocks * (kVecThreads / 32);
constexpr int kMaxGmresVecs = 128;


// ------------------------------------------------------------------------------------------
// argument blocks
// ------------------------------------------------------------------------------------------
struct LocalArgs {
  const SubMeta* meta;
  const int32_t *tnode_gid, *elem_gid, *lconn, *color_ptr, *rowptr, *colidx, *epos;
  const uint8_t* owned;
  double* csr;
  void* factor;
  void* dinv;  // packed triangular-solve operands (diagonal-block inverses + couplings)
  double* wbuf;
  double* work;        // three per-subdomain FP64 vectors (vec_off), `work_stride` apart
  int64_t work_stride;
  int32_t *its, *status;
  int32_t* chord;  // per subdomain: steps of the last launch taken with the stored factors
  int reuse;       // 1: a subdomain whose previous status is OK may start with chord steps
  const int32_t* order;
  int32_t* queue;
  const double *geom, *kcoef, *fext;
  double mu, lam, load;
  int ndof, nen, count, max_n, max_nt, max_b;
  double rtol, atol, armijo, ir_rtol;
  int maxit, ls_trials, ir_max;
  int l2_dist;            // L2 prefetch distance of the triangular solves (blocks; 0 = off)
  const double* x;        // evaluation point (global)
  double* out;            // F_x: owned entries receive x - w
  const double* guess;    // optional start states (concatenated local vectors)
  const double* guess_diag;  // Jacobi diagonal (leading term) of the smoothing of the start
  int guess_sweeps;
  double guess_omega;
  int want_tangent;
  int split_factor;           // 1: the tangent's band LU and packing run in k_local_factor
  int32_t* accepted;          // per subdomain: 1 where the proposed start was taken
  unsigned long long* phase;  // optional per-phase clock counters (profiling), see kPhaseNames
  // tangent application
  const double* v;
  const double* add;
  // coarse (harmonic extension / Galerkin)
  const double* phi;
  const int64_t* phi_off;
  const int32_t* cj_ptr;
  double* Y;
  double* blk;
  const int64_t* blk_off;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// shared-memory plan (bytes) of the local kernels
struct SmemPlan {
  size_t xt, r, rt, s, red, yv, win, rp, flag, total;
};

template <typename FT>
__host__ __device__ inline SmemPlan smem_plan(int max_n, int max_nt, int max_b, bool with_window) {
  SmemPlan p;
  size_t o = 0;
  p.xt = o; o += sizeof(double) * max_nt;
  p.r = o; o += sizeof(double) * max_n;
  p.rt = o; o += sizeof(double) * max_n;
  p.s = o; o += sizeof(double) * max_n;
  p.red = o; o += sizeof(double) * 40;
  p.yv = o; o += align_up(sizeof(FT) * max_n, 16);
  {
    const size_t lu = (size_t)dev::band_lu_window_rows(max_b) * dev::band_lu_window_stride(max_b);
    const size_t inv = 2 * (size_t)dev::SolveBlock<FT>::BS * (dev::SolveBlock<FT>::BS + 1);
    p.win = o;
    o += with_window ? align_up(sizeof(FT) * (lu > inv ? lu : inv), 16) : 0;
  }
  p.rp = o; o += with_window ? align_up(sizeof(FT) * dev::band_lu_window_rows(max_b), 16) : 0;
  p.flag = o; o += 16;
  p.total = o;
  return p;
}

// Shared memory of the batched local kernels.  Only what the inner loops hit per entry stays in
// shared memory -- the table state (gathered by every element), the residual being assembled,
// the band-LU window and the solve vector (which lives in the window once the factors are
// packed); the current residual, the Newton step and the refinement residual are per-subdomain
// vectors in global memory (read and written O(n) times per phase, coalesced).
struct LocalPlan {
  size_t xt, racc, red, win, rp, flag, total;
};

// Shared memory of the harmonic extension (k_harmonic): the table state, the solve vector and
// the window of dev::band_lu ((b + 2) rows of 2b + 1 entries, reciprocal pivots, flag), FP64.
__host__ __device__ inline SmemPlan harmonic_plan(int max_n, int max_nt, int max_b) {
  SmemPlan p;
  size_t o = 0;
  p.xt = o; o += align_up(sizeof(double) * max_nt, 16);
  p.r = p.rt = p.s = p.red = 0;  // unused
  p.yv = o; o += align_up(sizeof(double) * max_n, 16);
  p.win = o; o += align_up(sizeof(double) * (size_t)(max_b + 2) * (2 * max_b + 1), 16);
  p.rp = o; o += align_up(sizeof(double) * (max_b + 2), 16);
  p.flag = o; o += 16;
  p.total = o;
  return p;
}

template <typename FT>
__host__ __device__ inline LocalPlan newton_plan(int max_n, int max_nt, int max_b) {
  LocalPlan p;
  size_t o = 0;
  p.xt = o; o += sizeof(double) * max_nt;
  p.racc = o; o += sizeof(double) * max_n;
  p.red = o; o += sizeof(double) * 40;
  {
    const size_t lu = (size_t)dev::band_lu_window_rows(max_b) * dev::band_lu_window_stride(max_b);
    const size_t inv = 4 * (size_t)dev::SolveBlock<FT>::BS * (dev::SolveBlock<FT>::BS + 1);
    size_t w = lu > inv ? lu : inv;
    w = w > (size_t)max_n ? w : (size_t)max_n;
    p.win = o; o += align_up(sizeof(FT) * w, 16);
  }
  p.rp = o; o += align_up(sizeof(FT) * dev::band_lu_window_rows(max_b), 16);
  p.flag = o; o += 16;
  p.total = o;
  return p;
}

template <typename FT>
__host__ __device__ inline LocalPlan apply_plan(int max_n, int max_nt) {
  LocalPlan p;
  size_t o = 0;
  p.xt = o; o += sizeof(double) * max_nt;
  p.racc = 0;
  p.red = o; o += sizeof(double) * 40;
  p.win = o; o += align_up(sizeof(FT) * max_n, 16);
  p.rp = p.flag = o;
  p.total = o;
  return p;
}

// ------------------------------------------------------------------------------------------
// local assembly (colour-ordered, deterministic)
// ------------------------------------------------------------------------------------------
template <int LAW>
__device__ bool local_residual(const LocalArgs& A, const SubMeta& m, const double* xt, double* r) {
  const int nd = A.ndof, nen = A.nen;
  for (int a = threadIdx.x; a < m.n; a += blockDim.x) {
    const int64_t g = (int64_t)A.tnode_gid[m.tnode_off + a / nd] * nd + a % nd;
    r[a] = -A.load * A.fext[g];
  }
  __syncthreads();
  bool ok = true;
  const int32_t* cp = A.color_ptr + m.color_off;
  for (int c = 0; c < m.ncolor; ++c) {
    for (int e = cp[c] + threadIdx.x; e < cp[c + 1]; e += blockDim.x) {
      const int64_t le = m.elem_off + e;
      const int32_t gid = A.elem_gid[le];
      const int32_t* lc = A.lconn + le * nen;
      if (LAW == NLS_LAW_DIFFUSION) {
        const double* geo = A.geom + (int64_t)gid * 8;
        const dev::P1State st = dev::p1_state(geo, A.kcoef[gid], xt[lc[0]], xt[lc[1]], xt[lc[2]]);
        double re[3];
        dev::p1_residual(geo, st, re);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (lc[a] < m.nV) r[lc[a]] += re[a];
      } else {
        const double* geo = A.geom + (int64_t)gid * 40;
        double ue[8], re[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          ue[2 * a] = xt[2 * lc[a]];
          ue[2 * a + 1] = xt[2 * lc[a] + 1];
        }
        bool eok = true;
        dev::nh_residual(geo, ue, A.mu, A.lam, re, eok);
        ok = ok && eok;
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (lc[a] < m.nV) {
            r[2 * lc[a]] += re[2 * a];
            r[2 * lc[a] + 1] += re[2 * a + 1];
          }
      }
    }
    __syncthreads();
  }
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Local Jacobian into the CSR block of the subdomain (rows per m.nrows) and, when `band` is
// given, also into the band rows of the local matrix (row-major, 2 b + 1 per row, local
// unknowns only) that the in-place band LU then factors.  Element tangents are formed in FP64
// for both forms: the CSR block, against which the FP32 factors are refined, is the exact
// Jacobian; only the band copy that is factored is rounded to the factors' precision.
template <int LAW, typename FT = double>
__device__ void local_jacobian(const LocalArgs& A, const SubMeta& m, const double* xt, double* csr,
                               FT* band = nullptr) {
  const int nen = A.nen, nd = A.ndof, ned = nen * nd, ned2 = ned * ned;
  const int W = 2 * m.b + 1, n = m.n;
  for (int64_t k = threadIdx.x; k < m.nnz; k += blockDim.x) csr[k] = 0.0;
  if (band)
    for (int64_t k = threadIdx.x; k < (int64_t)n * W; k += blockDim.x) band[k] = (FT)0;
  __syncthreads();
  const int32_t* cp = A.color_ptr + m.color_off;
  for (int c = 0; c < m.ncolor; ++c) {
    for (int e = cp[c] + threadIdx.x; e < cp[c + 1]; e += blockDim.x) {
      const int64_t le = m.elem_off + e;
      const int32_t gid = A.elem_gid[le];
      const int32_t* lc = A.lconn + le * nen;
      const int32_t* ep = A.epos + m.epos_off + (int64_t)e * ned2;
      if (LAW == NLS_LAW_DIFFUSION) {
        const double* geo = A.geom + (int64_t)gid * 8;
        const dev::P1State st = dev::p1_state(geo, A.kcoef[gid], xt[lc[0]], xt[lc[1]], xt[lc[2]]);
        double K[9];
        dev::p1_jacobian<double>(geo, st, K);
        // the nine (row, col) targets of one element are distinct: issue every load before any
        // store so that one memory latency is paid per element, not one per entry
        double oc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) oc[q] = (ep[q] >= 0) ? csr[ep[q]] : 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q)
          if (ep[q] >= 0) csr[ep[q]] = oc[q] + K[q];
        if (band) {
          FT ob[9];
          int64_t bp[9];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              const bool in = lc[a] < n && lc[b] < n;
              bp[a * 3 + b] = in ? (int64_t)lc[a] * W + (lc[b] - lc[a] + m.b) : -1;
              ob[a * 3 + b] = in ? band[bp[a * 3 + b]] : (FT)0;
            }
#pragma unroll
          for (int q = 0; q < 9; ++q)
            if (bp[q] >= 0) band[bp[q]] = ob[q] + (FT)K[q];
        }
      } else {
        const double* geo = A.geom + (int64_t)gid * 40;
        double ue[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          ue[2 * a] = xt[2 * lc[a]];
          ue[2 * a + 1] = xt[2 * lc[a] + 1];
        }
        dev::NHGauss G;
        dev::nh_gauss(geo, ue, A.mu, A.lam, G);
#pragma unroll 1
        for (int a = 0; a < 4; ++a) {
          double R[16];
          dev::nh_tangent_rows(geo, G, A.mu, A.lam, a, R);
          const int32_t* epa = ep + 16 * a;  // rows (a, 0) and (a, 1): 16 consecutive targets
          double oc[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) oc[q] = (epa[q] >= 0) ? csr[epa[q]] : 0.0;
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (epa[q] >= 0) csr[epa[q]] = oc[q] + R[q];
          if (band && lc[a] < m.nV) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (lc[b] < m.nV) {
#pragma unroll
                for (int da = 0; da < 2; ++da)
#pragma unroll
                  for (int db = 0; db < 2; ++db) {
                    const int row = 2 * lc[a] + da, col = 2 * lc[b] + db;
                    band[(int64_t)row * W + (col - row + m.b)] += (FT)R[da * 8 + 2 * b + db];
                  }
              }
          }
        }
      }
    }
    __syncthreads();
  }
}

// s = J^-1 rhs with the band factors, then FP64 iterative refinement against the CSR matrix
// (columns < n) when the factors are FP32.  `res` is an n-vector of scratch.
template <typename FT, bool PF>
__device__ int local_solve(const LocalArgs& A, const SubMeta& m, const int32_t* rowptr, const int32_t* colidx,
                           const double* csr, const FT* Dv, const double* rhs, double rhs_norm, double* s,
                           double* res, FT* yv, double* red) {
  const int n = m.n;
  for (int a = threadIdx.x; a < n; a += blockDim.x) yv[a] = (FT)rhs[a];
  __syncthreads();
  dev::band_solve_packed<FT, PF>(n, m.b, Dv, yv, A.l2_dist);
  for (int a = threadIdx.x; a < n; a += blockDim.x) s[a] = (double)yv[a];
  __syncthreads();
  int sweeps = 0;
  if (sizeof(FT) == 4) {
    for (int sw = 0; sw < A.ir_max; ++sw) {
      double loc = 0.0;
      for (int a = threadIdx.x; a < n; a += blockDim.x) {
        double acc = rhs[a];
        for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) {
          const int col = colidx[k];
          if (col < n) acc -= csr[k] * s[col];
        }
        res[a] = acc;
        loc += acc * acc;
      }
      const double rn = sqrt(dev::block_sum(loc, red));
      if (!(rn > A.ir_rtol * rhs_norm)) break;
      for (int a = threadIdx.x; a < n; a += blockDim.x) yv[a] = (FT)res[a];
      __syncthreads();
      dev::band_solve_packed<FT, PF>(n, m.b, Dv, yv, A.l2_dist);
      for (int a = threadIdx.x; a < n; a += blockDim.x) s[a] += (double)yv[a];
      __syncthreads();
      ++sweeps;
    }
  }
  return sweeps;
}

// Damped Jacobi sweeps on a proposed local start (in xt's local unknowns): they remove the
// pointwise part of the proposal's error, w <- w - omega r(w) / (d (1 + w^2)) on all entries at
// once, d the diagonal of the Jacobian's leading term.  Leaves the residual of the result in racc
// and returns false if an evaluation was not finite.
template <int LAW>
__device__ bool smooth_proposal(const LocalArgs& A, const SubMeta& m, double* xt, double* racc) {
  bool okg = local_residual<LAW>(A, m, xt, racc);
  for (int sw = 0; sw < A.guess_sweeps && okg; ++sw) {
    for (int a = threadIdx.x; a < m.n; a += blockDim.x) {
      const double q = (LAW == NLS_LAW_DIFFUSION) ? 1.0 + xt[a] * xt[a] : 1.0;
      xt[a] -= A.guess_omega * racc[a] / (A.guess_diag[m.vec_off + a] * q);
    }
    __syncthreads();
    okg = local_residual<LAW>(A, m, xt, racc);
  }
  return okg;
}

// Test hook: the smoothing of given starts (A.guess, concatenated local vectors) at the point A.x,
// one CTA per subdomain, into A.out (concatenated local vectors).
template <int LAW>
__global__ void __launch_bounds__(256) k_guess_smooth(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* xt = (double*)smem;
  double* racc = xt + A.max_nt;
  const int sub = blockIdx.x, nd = A.ndof;
  const SubMeta m = A.meta[sub];
  for (int t = threadIdx.x; t < m.nt; t += blockDim.x)
    xt[t] = A.x[(int64_t)A.tnode_gid[m.tnode_off + t / nd] * nd + t % nd];
  __syncthreads();
  for (int a = threadIdx.x; a < m.n; a += blockDim.x) xt[a] = A.guess[m.vec_off + a];
  __syncthreads();
  smooth_proposal<LAW>(A, m, xt, racc);
  for (int a = threadIdx.x; a < m.n; a += blockDim.x) A.out[m.vec_off + a] = xt[a];
}

// ------------------------------------------------------------------------------------------
// k_local_newton: the batched local corrections T_i of Eq. 4
// ------------------------------------------------------------------------------------------
// MAXT is the largest CTA the instantiation is compiled for: 128-thread CTAs keep three CTAs
// per SM within the register file, 256-thread CTAs get the whole register budget per thread.
template <int LAW, typename FT, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 128 ? 4 : 1)) k_local_newton(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LocalPlan P = newton_plan<FT>(A.max_n, A.max_nt, A.max_b);
  double* xt = (double*)(smem + P.xt);
  double* racc = (double*)(smem + P.racc);  // residual being assembled
  double* red = (double*)(smem + P.red);
  FT* win = (FT*)(smem + P.win);
  FT* yv = win;  // the solve vector lives in the LU window once the factors are packed
  FT* rp = (FT*)(smem + P.rp);
  int* flag = (int*)(smem + P.flag);
  __shared__ int s_item;
  const int tid = threadIdx.x, nd = A.ndof;
  constexpr int BSI = dev::SolveBlock<FT>::BS;
  const int inv_warps = min((int)(blockDim.x >> 5), (int)((P.rp - P.win) / (sizeof(FT) * BSI * (BSI + 1))));
  long long tp = clock64();
  // thread 0 charges the cycles since the last mark to phase `id` (profiling only)
  auto mark = [&](int id) {
    if (A.phase && tid == 0) {
      const long long t = clock64();
      atomicAdd(A.phase + id, (unsigned long long)(t - tp));
      tp = t;
    }
  };
  for (;;) {
    if (tid == 0) s_item = atomicAdd(A.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= A.count) break;
    const int sub = A.order[item];
    const SubMeta m = A.meta[sub];
    const int n = m.n;
    const int32_t* rowptr = A.rowptr + m.rowptr_off;
    const int32_t* colidx = A.colidx + m.nnz_off;
    double* csr = A.csr + m.nnz_off;
    FT* F = (FT*)A.factor + m.factor_off;
    FT* Dv = (FT*)A.dinv + m.dinv_off;
    double* wb = A.wbuf + m.vec_off;
    double* r = A.work + m.vec_off;                            // current residual
    double* s = A.work + A.work_stride + m.vec_off;            // Newton step
    double* res = A.work + 2 * A.work_stride + m.vec_off;      // refinement residual
    for (int t = tid; t < m.nt; t += blockDim.x)
      xt[t] = A.x[(int64_t)A.tnode_gid[m.tnode_off + t / nd] * nd + t % nd];
    __syncthreads();
    bool ok = local_residual<LAW>(A, m, xt, racc);
    double loc = 0.0;
    for (int a = tid; a < n; a += blockDim.x) {
      r[a] = racc[a];
      loc += racc[a] * racc[a];
    }
    double rn = sqrt(dev::block_sum(loc, red));
    if (!ok) rn = INFINITY;
    // the stopping test is relative to the residual of the method's own start R_i x, with or
    // without a proposed start, so the proposal cannot change the accuracy of T_i
    const double tol = fmax(A.atol, A.rtol * rn);
    if (A.guess) {
      // acceptance test: take the proposed start only if its local residual is smaller
      for (int a = tid; a < n; a += blockDim.x) {
        wb[a] = xt[a];
        xt[a] = A.guess[m.vec_off + a];
      }
      __syncthreads();
      bool okg = smooth_proposal<LAW>(A, m, xt, racc);
      double lg = 0.0;
      for (int a = tid; a < n; a += blockDim.x) lg += racc[a] * racc[a];
      double rng = sqrt(dev::block_sum(lg, red));
      if (!okg) rng = INFINITY;
      const bool take = isfinite(rng) && rng < rn;
      if (take) {
        for (int a = tid; a < n; a += blockDim.x) r[a] = racc[a];
        rn = rng;
      } else {
        for (int a = tid; a < n; a += blockDim.x) xt[a] = wb[a];
      }
      __syncthreads();
      if (tid == 0 && A.accepted) A.accepted[sub] = take ? 1 : 0;
    }
    int its = 0, status = ST_OK, chord = 0;
    if (!isfinite(rn)) status = ST_NONFINITE;
    // the stored factors (and local Jacobian) are those of this subdomain's converged state of
    // the previous F_x evaluation when that evaluation succeeded here: chord steps with them
    // until one contracts the residual by less than a factor 10 or fails the line search
    bool stored = A.reuse && A.status[sub] == ST_OK;
    mark(0);
    while (status == ST_OK && rn > tol) {
      if (its >= A.maxit) {
        status = ST_MAXIT;
        break;
      }
      if (!stored) {
        local_jacobian<LAW, FT>(A, m, xt, csr, F);
        mark(1);
        if (dev::band_lu_inplace<FT>(n, m.b, F, win, rp, flag)) {
          status = ST_PIVOT;
          break;
        }
        dev::band_pack_solve<FT>(n, m.b, F, Dv, win, inv_warps);
        mark(2);
      }
      local_solve<FT, false>(A, m, rowptr, colidx, csr, Dv, r, rn, s, res, yv, red);
      mark(3);
      for (int a = tid; a < n; a += blockDim.x) wb[a] = xt[a];
      __syncthreads();
      double alpha = 1.0, rtn = INFINITY;
      bool accepted = false;
      for (int trial = 0; trial < A.ls_trials; ++trial) {
        for (int a = tid; a < n; a += blockDim.x) xt[a] = wb[a] - alpha * s[a];
        __syncthreads();
        const bool tok = local_residual<LAW>(A, m, xt, racc);
        double l2 = 0.0;
        for (int a = tid; a < n; a += blockDim.x) l2 += racc[a] * racc[a];
        rtn = sqrt(dev::block_sum(l2, red));
        if (!tok) rtn = INFINITY;
        if (isfinite(rtn) && rtn <= (1.0 - A.armijo * alpha) * rn) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      mark(4);
      if (!accepted) {
        for (int a = tid; a < n; a += blockDim.x) xt[a] = wb[a];
        __syncthreads();
        if (stored) {  // retry the step with the Jacobian at the current state
          stored = false;
          continue;
        }
        ++its;
        status = ST_LS;
        break;
      }
      ++its;
      if (stored) {
        ++chord;
        if (rtn > 0.1 * rn) stored = false;
      }
      for (int a = tid; a < n; a += blockDim.x) r[a] = racc[a];
      __syncthreads();
      rn = rtn;
    }
    if (A.want_tangent && status != ST_NONFINITE && status != ST_PIVOT) {
      local_jacobian<LAW, FT>(A, m, xt, csr, F);
      mark(5);
      if (!A.split_factor) {
        if (dev::band_lu_inplace<FT>(n, m.b, F, win, rp, flag)) status = ST_PIVOT;
        else dev::band_pack_solve<FT>(n, m.b, F, Dv, win, inv_warps);
      }
      mark(6);
    }
    for (int a = tid; a < n; a += blockDim.x) {
      wb[a] = xt[a];
      if (A.owned[m.vec_off + a]) {
        const int64_t g = (int64_t)A.tnode_gid[m.tnode_off + a / nd] * nd + a % nd;
        A.out[g] = A.x[g] - xt[a];
      }
    }
    if (tid == 0) {
      A.its[sub] = its;
      if (A.chord) A.chord[sub] = chord;
      A.status[sub] = status;
    }
    __syncthreads();
    mark(7);
  }
}

// ------------------------------------------------------------------------------------------
// k_local_factor: the tangent's refactorisation at the converged states -- band LU of the band
// that k_local_newton assembled and the packed solve operands -- as its own launch.  The Newton
// kernel's FP64 element tangents of Eq. 2 hold all of an SM's registers for one CTA; this kernel
// needs few registers and (FP32) about 65 KB of shared memory, so three CTAs share an SM and hide
// each other's per-step barrier latency.  One CTA per subdomain, longest first; subdomains whose
// local solve failed are skipped, a zero pivot marks the subdomain ST_PIVOT.
// ------------------------------------------------------------------------------------------
template <typename FT>
__host__ __device__ inline LocalPlan factor_plan(int max_b) {
  LocalPlan p{};
  size_t o = 0;
  const size_t lu = (size_t)dev::band_lu_window_rows(max_b) * dev::band_lu_window_stride(max_b);
  const size_t inv = 4 * (size_t)dev::SolveBlock<FT>::BS * (dev::SolveBlock<FT>::BS + 1);
  p.win = o; o += align_up(sizeof(FT) * (lu > inv ? lu : inv), 16);
  p.rp = o; o += align_up(sizeof(FT) * dev::band_lu_window_rows(max_b), 16);
  p.flag = o; o += 16;
  p.total = o;
  return p;
}

template <typename FT>
__global__ void __launch_bounds__(256, 3) k_local_factor(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LocalPlan P = factor_plan<FT>(A.max_b);
  FT* win = (FT*)(smem + P.win);
  FT* rp = (FT*)(smem + P.rp);
  int* flag = (int*)(smem + P.flag);
  constexpr int BSI = dev::SolveBlock<FT>::BS;
  const int inv_warps = min((int)(blockDim.x >> 5), (int)((P.rp - P.win) / (sizeof(FT) * BSI * (BSI + 1))));
  const int sub = A.order[blockIdx.x];
  const int st = A.status[sub];
  if (st == ST_NONFINITE || st == ST_PIVOT) return;
  const SubMeta m = A.meta[sub];
  FT* F = (FT*)A.factor + m.factor_off;
  FT* Dv = (FT*)A.dinv + m.dinv_off;
  if (dev::band_lu_inplace<FT>(m.n, m.b, F, win, rp, flag)) {
    if (threadIdx.x == 0) A.status[sub] = ST_PIVOT;
  } else {
    dev::band_pack_solve<FT>(m.n, m.b, F, Dv, win, inv_warps);
  }
}

// ------------------------------------------------------------------------------------------
// k_local_apply: out[owned] = (R_i DF(v_i) P_i)^-1 R_i DF(v_i) v  (+ add[owned])
// ------------------------------------------------------------------------------------------
template <typename FT>
__global__ void __launch_bounds__(512) k_local_apply(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LocalPlan P = apply_plan<FT>(A.max_n, A.max_nt);
  double* yt = (double*)(smem + P.xt);
  double* red = (double*)(smem + P.red);
  FT* yv = (FT*)(smem + P.win);
  const int sub = blockIdx.x, tid = threadIdx.x, nd = A.ndof;
  const SubMeta m = A.meta[sub];
  const int n = m.n;
  const int32_t* rowptr = A.rowptr + m.rowptr_off;
  const int32_t* colidx = A.colidx + m.nnz_off;
  const double* csr = A.csr + m.nnz_off;
  const FT* Dv = (const FT*)A.dinv + m.dinv_off;
  double* q = A.work + m.vec_off;
  double* z = A.work + A.work_stride + m.vec_off;
  double* res = A.work + 2 * A.work_stride + m.vec_off;
  for (int t = tid; t < m.nt; t += blockDim.x) yt[t] = A.v[(int64_t)A.tnode_gid[m.tnode_off + t / nd] * nd + t % nd];
  __syncthreads();
  double loc = 0.0;
  for (int a = tid; a < n; a += blockDim.x) {
    double acc = 0.0;
    for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) acc += csr[k] * yt[colidx[k]];
    q[a] = acc;
    loc += acc * acc;
  }
  const double qn = sqrt(dev::block_sum(loc, red));
  local_solve<FT, true>(A, m, rowptr, colidx, csr, Dv, q, qn, z, res, yv, red);
  for (int a = tid; a < n; a += blockDim.x)
    if (A.owned[m.vec_off + a]) {
      const int64_t g = (int64_t)A.tnode_gid[m.tnode_off + a / nd] * nd + a % nd;
      A.out[g] = z[a] + (A.add ? A.add[g] : 0.0);
    }
}

// ------------------------------------------------------------------------------------------
// coarse space: harmonic extension (setup) and Galerkin blocks
// ------------------------------------------------------------------------------------------
template <int LAW>
__global__ void __launch_bounds__(256) k_harmonic(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemPlan P = harmonic_plan(A.max_n, A.max_nt, A.max_b);
  double* xt = (double*)(smem + P.xt);
  double* yv = (double*)(smem + P.yv);
  double* win = (double*)(smem + P.win);
  double* rp = (double*)(smem + P.rp);
  int* flag = (int*)(smem + P.flag);
  const int j = blockIdx.x, tid = threadIdx.x, nd = A.ndof;
  const SubMeta m = A.meta[j];
  const int n = m.n;
  const int nc = A.cj_ptr[j + 1] - A.cj_ptr[j];
  double* phi = const_cast<double*>(A.phi) + A.phi_off[j];
  if (tid == 0) A.status[j] = ST_OK;
  const int32_t* rowptr = A.rowptr + m.rowptr_off;
  const int32_t* colidx = A.colidx + m.nnz_off;
  double* csr = A.csr + m.nnz_off;
  double* F = (double*)A.factor + m.factor_off;
  for (int t = tid; t < m.nt; t += blockDim.x) xt[t] = A.x[(int64_t)A.tnode_gid[m.tnode_off + t / nd] * nd + t % nd];
  __syncthreads();
  local_jacobian<LAW>(A, m, xt, csr);
  if (n == 0 || nc == 0) return;
  dev::RowSource src{rowptr, colidx, csr};
  if (dev::band_lu<double>(n, m.b, src, F, win, rp, flag)) {
    if (tid == 0) A.status[j] = ST_PIVOT;
    return;
  }
  for (int lc = 0; lc < nc; ++lc) {
    for (int a = tid; a < n; a += blockDim.x) {
      double acc = 0.0;
      for (int k = rowptr[a]; k < rowptr[a + 1]; ++k) {
        const int col = colidx[k];
        if (col >= n) acc -= csr[k] * phi[(int64_t)col * nc + lc];
      }
      yv[a] = acc;
    }
    __syncthreads();
    dev::band_solve<double>(n, m.b, F, yv);
    for (int a = tid; a < n; a += blockDim.x) phi[(int64_t)a * nc + lc] = yv[a];
    __syncthreads();
  }
}

template <int LAW>
__global__ void __launch_bounds__(256) k_galerkin(LocalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemPlan P = smem_plan<double>(A.max_n, A.max_nt, A.max_b, false);
  double* xt = (double*)(smem + P.xt);
  const int j = blockIdx.x, tid = threadIdx.x, nd = A.ndof;
  const SubMeta m = A.meta[j];
  const int nc = A.cj_ptr[j + 1] - A.cj_ptr[j];
  const double* phi = A.phi + A.phi_off[j];
  double* Y = A.Y + A.phi_off[j];
  const int32_t* rowptr = A.rowptr + m.rowptr_off;
  const int32_t* colidx = A.colidx + m.nnz_off;
  double* csr = A.csr + m.nnz_off;
  for (int t = tid; t < m.nt; t += blockDim.x) xt[t] = A.x[(int64_t)A.tnode_gid[m.tnode_off + t / nd] * nd + t % nd];
  __syncthreads();
  local_jacobian<LAW>(A, m, xt, csr);
  if (nc == 0) return;
  // Y = K^(j) Phi_j
  for (int64_t idx = tid; idx < (int64_t)m.nt * nc; idx += blockDim.x) {
    const int t = (int)(idx / nc), lc = (int)(idx % nc);
    double acc = 0.0;
    for (int k = rowptr[t]; k < rowptr[t + 1]; ++k) acc += csr[k] * phi[(int64_t)colidx[k] * nc + lc];
    Y[idx] = acc;
  }
  __syncthreads();
  // block = Phi_j^T Y, one warp per entry, fixed-order lane sums
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  double* blk = A.blk + A.blk_off[j];
  for (int e = wid; e < nc * nc; e += nw) {
    const int c = e / nc, d = e % nc;
    double acc = 0.0;
    for (int t = lane; t < m.nt; t += 32) acc += phi[(int64_t)t * nc + c] * Y[(int64_t)t * nc + d];
    acc = dev::warp_sum(acc);
    if (lane == 0) blk[e] = acc;
  }
}

__global__ void k_a0_gather(int64_t nentries, const int32_t* ptr, const int64_t* src, const double* blk, double* A0) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nentries; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int32_t k = ptr[e]; k < ptr[e + 1]; ++k) acc += blk[src[k]];
    A0[e] = acc;
  }
}

__global__ void k_gather_values(int64_t n, const int64_t* src, const double* from, double* to) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    to[k] = from[src[k]];
}

__global__ void k_gather_values32(int64_t n, const int32_t* src, const double* from, double* to) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    to[k] = from[src[k]];
}

// coarse band factorization (one CTA)
template <typename FT>
__global__ void __launch_bounds__(1024) k_coarse_factor(int N0, int b0, const double* A0, FT* F, FT* Dinv, int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int BS = dev::SolveBlock<FT>::BS;
  const size_t R = (size_t)dev::band_lu_window_rows(b0);
  FT* win = (FT*)smem;
  FT* rp = win + R * dev::band_lu_window_stride(b0);
  FT* tmp = rp + R;
  int* flag = (int*)(tmp + 4 * BS * (BS + 1));
  const int64_t total = (int64_t)N0 * (2 * b0 + 1);
  for (int64_t k = threadIdx.x; k < total; k += blockDim.x) F[k] = (FT)A0[k];
  __syncthreads();
  const int bad = dev::band_lu_inplace<FT>(N0, b0, F, win, rp, flag);
  // the LU window is free again: it holds the packing scratch of up to every warp
  const int pw = min((int)(blockDim.x >> 5), (int)((R * dev::band_lu_window_stride(b0)) / (BS * (BS + 1))));
  if (!bad) dev::band_pack_solve<FT>(N0, b0, F, Dinv, pw >= 4 ? win : tmp, pw >= 4 ? pw : 4);
  if (threadIdx.x == 0) *status = bad ? ST_PIVOT : ST_OK;
}

// Columns of A_0^-1 from the band factors (one CTA per column, the solve vector in shared
// memory): one solve A_0 z = e_col in the factors' precision (the forward sweep starts at the
// block of `col`, above which e_col and z vanish), stored in that precision and transposed
// (AinvT[col][row]) so that the GEMV below reads it coalesced.  FP32 columns are refined where
// they are applied (coarse_solve): the FP64 residual of one vector costs N0 (2 b0 + 1)
// multiply-adds, that of every column of the inverse N0 times as many.
template <typename FT>
__global__ void __launch_bounds__(512) k_coarse_inverse(int N0, int b0, const FT* Dinv, FT* AinvT, int l2d) {
  extern __shared__ __align__(16) unsigned char smem[];
  FT* y = (FT*)smem;
  constexpr int BS = dev::SolveBlock<FT>::BS;
  for (int col = blockIdx.x; col < N0; col += gridDim.x) {
    for (int a = threadIdx.x; a < N0; a += blockDim.x) y[a] = (a == col) ? (FT)1 : (FT)0;
    __syncthreads();
    dev::band_solve_packed<FT, false>(N0, b0, Dinv, y, l2d, col / BS);
    for (int a = threadIdx.x; a < N0; a += blockDim.x) AinvT[(int64_t)col * N0 + a] = y[a];
    __syncthreads();
  }
}

// z = A_0^-1 g with the explicit inverse (stored transposed).  Grid (row tiles of 32, column
// chunks): lane = row, the 8 warps of a CTA stride over the chunk's columns (coalesced rows of
// AinvT), warp partials are summed in shared memory in warp order, chunk partials go to
// `part` and k_gemv_finish adds them in chunk order (no atomics: the result is reproducible).
// With `skip` set (a refinement that has converged) both kernels return at once.
constexpr int kGemvChunks = 16;
// Largest coarse dimension with an explicit inverse (N0^2 entries in the factors' precision:
// 1 GB in FP32 at the limit); larger coarse problems use the one-CTA band solve.
constexpr int kMaxInverseN0 = 16384;
template <typename FT>
__global__ void __launch_bounds__(256) k_dense_gemv_t(int N0, const FT* AinvT, const double* g, double* part,
                                                       const int* skip) {
  if (skip && *skip) return;
  __shared__ double acc_s[8][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + lane;
  const int per = (N0 + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(N0, c0 + per);
  double acc = 0.0;
  if (row < N0)
    for (int col = c0 + wid; col < c1; col += 8) acc += (double)AinvT[(int64_t)col * N0 + row] * g[col];
  acc_s[wid][lane] = acc;
  __syncthreads();
  if (wid == 0 && row < N0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += acc_s[w][lane];
    part[(int64_t)blockIdx.y * N0 + row] = t;
  }
}

// z = sum of the chunk partials (accumulate = 0) or z += it (accumulate = 1); `reset`, if
// given, is cleared (the refinement flag of the solve that starts here).
__global__ void k_gemv_finish(int N0, int chunks, const double* part, double* z, int accumulate, const int* skip,
                              int* reset) {
  if (skip && *skip) return;
  if (reset && blockIdx.x == 0 && threadIdx.x == 0) *reset = 0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N0; row += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += part[(int64_t)c * N0 + row];
    z[row] = accumulate ? z[row] + t : t;
  }
}

// One step of the refinement of an explicit-inverse coarse solve: r = g - A_0 z (FP64 band
// A_0, one warp per row, 8 rows per CTA) and its test.  Every CTA stores its partial sums of
// r^2 and g^2; the last CTA to finish (atomic ticket) adds them in CTA order and sets *done
// when ||r|| <= ir_rtol ||g|| (or the norms are not finite), then returns the ticket counter
// to 0.  With *done already set the kernel does nothing.
__global__ void __launch_bounds__(256) k_coarse_residual(int N0, int b0, const double* A0, const double* g,
                                                          const double* z, double* r, double* part,
                                                          unsigned* ticket, int* done, double ir_rtol) {
  if (*done) return;
  __shared__ double s_r[8], s_g[8];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int a = blockIdx.x * 8 + wid, W = 2 * b0 + 1;
  double rr = 0.0, gg = 0.0;
  if (a < N0) {
    double acc = 0.0;
    for (int d = lane; d < W; d += 32) {
      const int cc = a - b0 + d;
      if (cc >= 0 && cc < N0) acc += A0[(int64_t)a * W + d] * z[cc];
    }
    acc = dev::warp_sum(acc);
    const double ra = g[a] - acc;
    if (lane == 0) r[a] = ra;
    rr = ra * ra;
    gg = g[a] * g[a];
  }
  if (lane == 0) s_r[wid] = rr, s_g[wid] = gg;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tg = 0.0;
    for (int w = 0; w < 8; ++w) tr += s_r[w], tg += s_g[w];
    part[2 * blockIdx.x] = tr;
    part[2 * blockIdx.x + 1] = tg;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && wid == 0) {
    __threadfence();
    double tr = 0.0, tg = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) tr += __ldcg(part + 2 * b), tg += __ldcg(part + 2 * b + 1);
    tr = dev::warp_sum(tr);
    tg = dev::warp_sum(tg);
    if (lane == 0) {
      *done = !(sqrt(tr) > ir_rtol * sqrt(tg)) ? 1 : 0;
      *ticket = 0;
    }
  }
}

// One coarse solve with the packed band factors in one CTA (the solve vector in shared memory):
// z = (accumulate ? z : 0) + A_0^-1 rhs in the factors' precision.  With *skip set (a refinement
// that has converged) the kernel does nothing; `reset`, if given, is cleared (the refinement flag
// of the solve that starts here).  Needs blockDim.x >= 32 + b0.
template <typename FT>
__global__ void __launch_bounds__(512) k_coarse_band_solve(int N0, int b0, const FT* Dinv, const double* rhs,
                                                             double* z, int accumulate, const int* skip, int* reset,
                                                             int l2d) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem[];
  FT* y = (FT*)smem;
  if (reset && threadIdx.x == 0) *reset = 0;
  for (int a = threadIdx.x; a < N0; a += blockDim.x) y[a] = (FT)rhs[a];
  __syncthreads();
  dev::band_solve_packed<FT, true>(N0, b0, Dinv, y, l2d);
  for (int a = threadIdx.x; a < N0; a += blockDim.x) z[a] = (accumulate ? z[a] : 0.0) + (double)y[a];
}

// ------------------------------------------------------------------------------------------
// global assembly: the residual by element contributions and node sums, the Jacobian in colour
// passes (elements of one colour share no node)
// ------------------------------------------------------------------------------------------
// Element residuals (the weak forms of Eqs. 1 and 2) of every element, one thread per element,
// into Re[(e nen + a) ndof + d]; k_node_residual adds them up per node.
template <int LAW>
__global__ void k_elem_residual(int64_t ne, const int32_t* conn, const double* geom, const double* kcoef,
                                const double* x, double* Re, double mu, double lam, int* bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    if (LAW == NLS_LAW_DIFFUSION) {
      const int32_t* c = conn + e * 3;
      const double* geo = geom + e * 8;
      const dev::P1State st = dev::p1_state(geo, kcoef[e], x[c[0]], x[c[1]], x[c[2]]);
      double re[3];
      dev::p1_residual(geo, st, re);
#pragma unroll
      for (int a = 0; a < 3; ++a) Re[e * 3 + a] = re[a];
    } else {
      const int32_t* c = conn + e * 4;
      const double* geo = geom + e * 40;
      double ue[8], re[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ue[2 * a] = x[2 * (int64_t)c[a]];
        ue[2 * a + 1] = x[2 * (int64_t)c[a] + 1];
      }
      bool ok = true;
      dev::nh_residual(geo, ue, mu, lam, re, ok);
      if (!ok) *bad = 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) Re[e * 8 + q] = re[q];
    }
  }
}

// F = -load fext + the contributions of the elements around every node, added in ascending
// element order (star_ref[k] = e nen + a: element e, where the node is e's a-th); 0 on the
// Dirichlet dofs.
__global__ void k_node_residual(int64_t n_nodes, int nd, const int64_t* star_ptr, const int32_t* star_ref,
                                const double* Re, double load, const double* fext, const uint8_t* free_dof,
                                double* F) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes;
       v += (int64_t)gridDim.x * blockDim.x) {
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t k = star_ptr[v]; k < star_ptr[v + 1]; ++k) {
      const int64_t r = (int64_t)star_ref[k] * nd;
      acc0 += Re[r];
      if (nd == 2) acc1 += Re[r + 1];
    }
    for (int d = 0; d < nd; ++d) {
      const int64_t i = v * nd + d;
      F[i] = free_dof[i] ? -load * fext[i] + (d == 0 ? acc0 : acc1) : 0.0;
    }
  }
}

template <int LAW>
__global__ void k_global_jacobian(const int32_t* elems, int e0, int e1, const int32_t* conn, const double* geom,
                                  const double* kcoef, const double* x, const int32_t* epos, double* val, double mu,
                                  double lam) {
  for (int i = e0 + blockIdx.x * blockDim.x + threadIdx.x; i < e1; i += gridDim.x * blockDim.x) {
    const int32_t e = elems[i];
    if (LAW == NLS_LAW_DIFFUSION) {
      const int32_t* c = conn + (int64_t)e * 3;
      const double* geo = geom + (int64_t)e * 8;
      const dev::P1State st = dev::p1_state(geo, kcoef[e], x[c[0]], x[c[1]], x[c[2]]);
      double K[9];
      dev::p1_jacobian<double>(geo, st, K);
      const int32_t* ep = epos + (int64_t)e * 9;
#pragma unroll
      for (int q = 0; q < 9; ++q) val[ep[q]] += K[q];
    } else {
      const int32_t* c = conn + (int64_t)e * 4;
      const double* geo = geom + (int64_t)e * 40;
      double ue[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ue[2 * a] = x[2 * (int64_t)c[a]];
        ue[2 * a + 1] = x[2 * (int64_t)c[a] + 1];
      }
      dev::NHGauss G;
      dev::nh_gauss(geo, ue, mu, lam, G);
      const int32_t* ep = epos + (int64_t)e * 64;
#pragma unroll 1
      for (int a = 0; a < 4; ++a) {
        double R[16];
        dev::nh_tangent_rows(geo, G, mu, lam, a, R);
#pragma unroll
        for (int q = 0; q < 16; ++q) val[ep[16 * a + q]] += R[q];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// vector kernels
// ------------------------------------------------------------------------------------------
__global__ void k_axpby(int64_t n, double a, const double* x, double b, const double* y, double* z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

__global__ void k_mask(int64_t n, const uint8_t* free_dof, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!free_dof[i]) x[i] = 0.0;
}

__global__ void k_set_dirichlet(int64_t n, const uint8_t* free_dof, const double* ubc, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!free_dof[i]) x[i] = ubc[i];
}

// y = J x on free rows (0 on Dirichlet rows)
__global__ void k_spmv_free(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                            const uint8_t* free_dof, const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (free_dof[i])
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += val[k] * x[col[k]];
    y[i] = acc;
  }
}

// y = a * x + s * (P0 c)
__global__ void k_p0_apply(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* c,
                           double a, const double* x, double s, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += val[k] * c[col[k]];
    y[i] = (x ? a * x[i] : 0.0) + s * acc;
  }
}

// g = P0^T v, one CTA per coarse row (the rows are long: every fine dof in the support of the
// coarse function); fixed-order warp and CTA sums.
__global__ void __launch_bounds__(256) k_p0t_apply(int n0, const int32_t* rowptr, const int32_t* col,
                                                    const double* val, const double* v, double* g) {
  __shared__ double red[40];
  for (int r = blockIdx.x; r < n0; r += gridDim.x) {
    double acc = 0.0;
    for (int32_t k = rowptr[r] + threadIdx.x; k < rowptr[r + 1]; k += blockDim.x) acc += val[k] * v[col[k]];
    acc = dev::block_sum(acc, red);
    if (threadIdx.x == 0) g[r] = acc;
  }
}

// per-warp partial dot products of `nv` vectors (stride ld) with w
__global__ void k_multidot_partial(int64_t n, int nv, const double* V, int64_t ld, const double* w, double* partial) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int i = 0; i < nv; ++i) {
    const double* vi = V + (int64_t)i * ld;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) acc += vi[k] * w[k];
    acc = dev::warp_sum(acc);
    if (lane == 0) partial[(int64_t)i * kVecWarps + gw] = acc;
  }
}

__global__ void k_partial_final(int nv, const double* partial, double* out) {
  __shared__ double red[40];
  for (int i = blockIdx.x; i < nv; i += gridDim.x) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < kVecWarps; k += blockDim.x) acc += partial[(int64_t)i * kVecWarps + k];
    acc = dev::block_sum(acc, red);
    if (threadIdx.x == 0) out[i] = acc;
    __syncthreads();
  }
}

// w -= sum_i coef[i] V_i
__global__ void k_multiaxpy(int64_t n, int nv, const double* V, int64_t ld, const double* coef, double sign, double* w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nv; ++i) acc += coef[i] * V[(int64_t)i * ld + k];
    w[k] += sign * acc;
  }
}

__global__ void k_scale_inv(int64_t n, const double* x, const double* nrm, double* y) {
  const double s = 1.0 / *nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}

__global__ void k_sqrt_inplace(double* x) { *x = sqrt(*x); }

// ---- GMRES least-squares state on the device (GmresState) --------------------------------------

// A new cycle: g = (rn, 0, ..., 0).
__global__ void k_gmres_start(int m, double rn, double target, int limit, double* g, GmresState* st) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? rn : 0.0;
  if (threadIdx.x == 0) {
    st->j = 0;
    st->done = 0;
    st->limit = limit;
    st->target = target;
    st->res = rn;
  }
}

// After iteration j: the Hessenberg column h_i = scal[i] + scal[half + i] (the two Gram-Schmidt
// passes, i <= j) and h_{j+1} = scal[kMaxGmresVecs]; apply the earlier rotations to it, form the
// rotation that annihilates h_{j+1}, rotate g, keep the column of R (row-major, m x m); then
// decide whether the cycle goes on, and (inside a graph) set `h`, the condition of the next
// iteration's IF node.
__global__ void k_gmres_givens(int j, int m, const double* scal, double* Rm, double* cs, double* sn, double* g,
                               GmresState* st, cudaGraphConditionalHandle h, int use_handle) {
  if (threadIdx.x != 0) return;
  double col[kMaxGmresVecs / 2 + 1];
  for (int i = 0; i <= j; ++i) col[i] = scal[i] + scal[kMaxGmresVecs / 2 + i];
  const double hn = scal[kMaxGmresVecs];
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double d = hypot(col[j], hn);
  cs[j] = col[j] / d;
  sn[j] = hn / d;
  col[j] = d;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  for (int i = 0; i <= j; ++i) Rm[(size_t)i * m + j] = col[i];
  const double res = fabs(g[j + 1]);
  const int done = (!isfinite(hn) || res <= st->target || hn == 0.0) ? 1 : 0;
  st->j = j + 1;
  st->res = res;
  st->done = done;
  if (use_handle) cudaGraphSetConditional(h, (!done && j + 1 < st->limit) ? 1u : 0u);
}

// y = R^-1 g over the cycle's st->j iterations (back substitution) into coef.
__global__ void k_gmres_lsq(int m, const double* Rm, const double* g, const GmresState* st, double* coef) {
  if (threadIdx.x != 0) return;
  const int n = st->j;
  for (int i = n - 1; i >= 0; --i) {
    double acc = g[i];
    for (int k = i + 1; k < n; ++k) acc -= Rm[(size_t)i * m + k] * coef[k];
    coef[i] = acc / Rm[(size_t)i * m + i];
  }
}

// w += sign sum_{i < st->j} coef[i] V_i (the number of vectors read from the device)
__global__ void k_multiaxpy_dev(int64_t n, const GmresState* st, const double* V, int64_t ld, const double* coef,
                                double sign, double* w) {
  const int nv = st->j;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nv; ++i) acc += coef[i] * V[(int64_t)i * ld + k];
    w[k] += sign * acc;
  }
}

}  // namespace


namespace {

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, kVecBlocks));
}


// The triangular solves need warp 0 plus one thread per coupled row (32 + b threads).
int min_local_threads(const Context& c) { return ((32 + c.ov.max_b + 31) / 32) * 32; }

int local_threads(const Context& c) {
  int pick = c.opt.threads_per_block ? c.opt.threads_per_block : (c.ndof == 1 ? 128 : 256);
  if (!c.opt.threads_per_block && c.dev && c.dev->newton_T) pick = c.dev->newton_T;
  return std::max(pick, min_local_threads(c));
}

int apply_threads(const Context& c) {
  if (c.dev && c.dev->apply_T) return std::max(c.dev->apply_T, min_local_threads(c));
  return std::max(64, min_local_threads(c));
}

bool fp32_local(const Context& c) { return c.opt.local_precision == NLS_PREC_FP32_IR; }
bool fp32_coarse(const Context& c) { return c.opt.coarse_precision == NLS_PREC_FP32_IR; }

// Largest half bandwidth of A_0 the one-CTA band LU takes (its window sits in shared memory) and
// that the coarse band solves take (warp 0 plus one thread per coupled row in a CTA of at most
// 512 threads, which keeps 128 registers per thread for the double-buffered operands).
constexpr int kMaxBandB0 = 128;
constexpr int kMaxSolveB0 = 512 - 32;

bool coarse_tiles(const Context& c) {
  return c.opt.coarse_factor == NLS_COARSE_FACTOR_TILES ||
         (c.opt.coarse_factor == NLS_COARSE_FACTOR_AUTO && c.cs.b0 > kMaxBandB0);
}

// CTA size of the one-CTA coarse band solves: warp 0 plus one thread per coupled row.
int coarse_solve_threads(const Context& c) { return std::max(256, (32 + c.cs.b0 + 31) / 32 * 32); }

LocalArgs make_args(const Context& c, const LocalSet& hs, const DeviceLocalSet& ds) {
  LocalArgs A;
  std::memset(&A, 0, sizeof(A));
  Dev& D = *c.dev;
  A.meta = ds.meta;
  A.tnode_gid = ds.tnode_gid;
  A.elem_gid = ds.elem_gid;
  A.lconn = ds.lconn;
  A.color_ptr = ds.color_ptr;
  A.rowptr = ds.rowptr;
  A.colidx = ds.colidx;
  A.epos = ds.epos;
  A.owned = ds.owned;
  A.csr = ds.csr_val;
  A.factor = ds.factor;
  A.dinv = ds.dinv;
  A.wbuf = ds.w;
  A.work = ds.work;
  A.work_stride = hs.total_n;
  A.its = ds.its;
  A.status = ds.status;
  A.chord = ds.chord;
  A.reuse = 0;
  A.order = ds.order;
  A.queue = ds.queue;
  A.geom = D.geom;
  A.kcoef = D.kcoef;
  A.fext = D.fext;
  lame(c, A.mu, A.lam);
  A.load = 1.0;
  A.ndof = c.ndof;
  A.nen = c.nen;
  A.count = hs.count;
  A.max_n = hs.max_n;
  A.max_nt = hs.max_nt;
  A.max_b = hs.max_b;
  A.rtol = c.opt.inner_rtol;
  A.atol = c.opt.inner_atol;
  A.armijo = c.opt.armijo;
  A.ir_rtol = c.opt.ir_rtol;
  A.maxit = c.opt.inner_maxit;
  A.ls_trials = c.opt.ls_trials;
  A.ir_max = c.opt.ir_max_sweeps;
  A.l2_dist = c.opt.l2_prefetch;
  return A;
}

// Allow the kernel the whole opt-in shared memory minus its static shared memory.
template <typename K>
void set_smem(K kernel, size_t optin) {
  cudaFuncAttributes fa;
  CK(cudaFuncGetAttributes(&fa, kernel));
  const size_t dyn = optin > fa.sharedSizeBytes ? optin - fa.sharedSizeBytes : 0;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
}

void sync(Dev& D) { CK(cudaStreamSynchronize(D.s)); }

// ---- reductions with a host read-back ---------------------------------------------------------
double dot(Dev& D, int64_t n, const double* x, const double* y) {
  LAUNCH(D, k_multidot_partial, kVecBlocks, kVecThreads, 0, n, 1, x, (int64_t)0, y, D.partial);
  LAUNCH(D, k_partial_final, 1, 256, 0, 1, D.partial, D.scal);
  CK(cudaMemcpyAsync(D.h_scal, D.scal, sizeof(double), cudaMemcpyDeviceToHost, D.s));
  sync(D);
  return D.h_scal[0];
}

// A NaN or infinite sum of squares stays non-finite (std::max(0.0, NaN) would give 0: a NaN state
// must never read as converged).
double norm2(Dev& D, int64_t n, const double* x) {
  const double d = dot(D, n, x, x);
  return std::isfinite(d) ? std::sqrt(std::max(0.0, d)) : d;
}

// ---- global residual / Jacobian ------------------------------------------------------------
void global_residual(Context& c, const double* x, double* F, double load) {
  Dev& D = *c.dev;
  double mu, lam;
  lame(c, mu, lam);
  if (c.law == NLS_LAW_DIFFUSION)
    LAUNCH(D, k_elem_residual<NLS_LAW_DIFFUSION>, grid_for(c.n_elems), 256, 0, c.n_elems, D.conn, D.geom, D.kcoef, x,
           D.Re, mu, lam, D.bad);
  else
    LAUNCH(D, k_elem_residual<NLS_LAW_NEOHOOKE>, grid_for(c.n_elems), 256, 0, c.n_elems, D.conn, D.geom, D.kcoef, x,
           D.Re, mu, lam, D.bad);
  LAUNCH(D, k_node_residual, grid_for(c.n_nodes), 256, 0, c.n_nodes, c.ndof, D.star_ptr, D.star_ref, D.Re, load,
         D.fext, D.free_dof, F);
}

void global_jacobian(Context& c, const double* x) {
  Dev& D = *c.dev;
  double mu, lam;
  lame(c, mu, lam);
  CK(cudaMemsetAsync(D.g_val, 0, sizeof(double) * c.g_col.size(), D.s));
  for (size_t k = 0; k + 1 < c.g_color_ptr.size(); ++k) {
    const int e0 = c.g_color_ptr[k], e1 = c.g_color_ptr[k + 1];
    if (c.law == NLS_LAW_DIFFUSION)
      LAUNCH(D, (k_global_jacobian<NLS_LAW_DIFFUSION>), grid_for(e1 - e0), 256, 0, D.g_elem, e0, e1, D.conn, D.geom,
             D.kcoef, x, D.g_epos, D.g_val, mu, lam);
    else
      LAUNCH(D, (k_global_jacobian<NLS_LAW_NEOHOOKE>), grid_for(e1 - e0), 256, 0, D.g_elem, e0, e1, D.conn, D.geom,
             D.kcoef, x, D.g_epos, D.g_val, mu, lam);
  }
}

// ---- batched local kernels ---------------------------------------------------------------------
template <typename FT>
size_t local_newton_smem(const LocalSet& s) {
  return newton_plan<FT>(s.max_n, s.max_nt, s.max_b).total;
}

// Persistent grid: as many CTAs as fit on the device at once (registers and shared memory), at
// most one per subdomain; the work counter hands out the subdomains.
const char* newton_kernel_name(int law, bool f32, int maxt) {
  static const char* names[8] = {
      "k_local_newton<diffusion, double, 128>", "k_local_newton<diffusion, float, 128>",
      "k_local_newton<diffusion, double, 256>", "k_local_newton<diffusion, float, 256>",
      "k_local_newton<neohooke, double, 128>",  "k_local_newton<neohooke, float, 128>",
      "k_local_newton<neohooke, double, 256>",  "k_local_newton<neohooke, float, 256>"};
  return names[(law == NLS_LAW_DIFFUSION ? 0 : 4) + (maxt > 128 ? 2 : 0) + (f32 ? 1 : 0)];
}

template <int LAW, typename FT, int MAXT>
void launch_newton_t(Dev& D, int count, int T, size_t sm, const LocalArgs& A) {
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_newton<LAW, FT, MAXT>, T, sm));
  occ = std::max(1, occ);
  // With one CTA per SM a concurrent one-CTA coarse factorization could never share an SM with
  // this persistent grid: leave it one (the CTAs pull subdomains from the work counter, so one
  // fewer CTA only means more subdomains for the others).
  const int spare = (D.coarse_beside && occ == 1 && D.nsm > 1) ? 1 : 0;
  const int grid = std::min(count, (D.nsm - spare) * occ);
  LAUNCH_NAMED(D, newton_kernel_name(LAW, sizeof(FT) == 4, MAXT), (k_local_newton<LAW, FT, MAXT>), grid, T, sm, A);
}

template <int LAW, typename FT>
void launch_newton_law(Dev& D, int count, int T, size_t sm, const LocalArgs& A) {
  if (T <= 128) launch_newton_t<LAW, FT, 128>(D, count, T, sm, A);
  else launch_newton_t<LAW, FT, 256>(D, count, T, sm, A);
}

// CTAs of the batched local Newton kernel resident per SM at the current CTA size.
int newton_ctas_per_sm(Context& c) {
  const int T = local_threads(c);
  const bool f32 = fp32_local(c);
  const size_t sm = f32 ? local_newton_smem<float>(c.ov) : local_newton_smem<double>(c.ov);
  int occ = 0;
  auto q = [&](auto kernel) { CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, T, sm)); };
  const bool big = T > 128;
  if (c.law == NLS_LAW_DIFFUSION) {
    if (f32) big ? q(k_local_newton<NLS_LAW_DIFFUSION, float, 256>) : q(k_local_newton<NLS_LAW_DIFFUSION, float, 128>);
    else big ? q(k_local_newton<NLS_LAW_DIFFUSION, double, 256>) : q(k_local_newton<NLS_LAW_DIFFUSION, double, 128>);
  } else {
    if (f32) big ? q(k_local_newton<NLS_LAW_NEOHOOKE, float, 256>) : q(k_local_newton<NLS_LAW_NEOHOOKE, float, 128>);
    else big ? q(k_local_newton<NLS_LAW_NEOHOOKE, double, 256>) : q(k_local_newton<NLS_LAW_NEOHOOKE, double, 128>);
  }
  return std::max(1, occ);
}

// The tangent's refactorisation goes to k_local_factor when the Newton kernel, at its current
// CTA size, holds one CTA per SM and the factor kernel fits at least two.
bool split_local_factor(Context& c) {
  int occ = 0;
  if (fp32_local(c))
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_factor<float>, 256, factor_plan<float>(c.ov.max_b).total));
  else
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_factor<double>, 256, factor_plan<double>(c.ov.max_b).total));
  return newton_ctas_per_sm(c) == 1 && occ >= 2;
}

void dispatch_local_newton(Context& c, const LocalSet& s, const LocalArgs& A, int T) {
  Dev& D = *c.dev;
  const bool f32 = fp32_local(c);
  const size_t sm = f32 ? local_newton_smem<float>(s) : local_newton_smem<double>(s);
  if (c.law == NLS_LAW_DIFFUSION) {
    if (f32) launch_newton_law<NLS_LAW_DIFFUSION, float>(D, s.count, T, sm, A);
    else launch_newton_law<NLS_LAW_DIFFUSION, double>(D, s.count, T, sm, A);
  } else {
    if (f32) launch_newton_law<NLS_LAW_NEOHOOKE, float>(D, s.count, T, sm, A);
    else launch_newton_law<NLS_LAW_NEOHOOKE, double>(D, s.count, T, sm, A);
  }
}

void launch_local_newton(Context& c, const double* x, double* out, double load, const GuessProposal& g,
                         bool want_tangent) {
  Dev& D = *c.dev;
  LocalArgs A = make_args(c, c.ov, D.ov);
  A.x = x;
  A.out = out;
  A.load = load;
  A.guess = g.x;
  A.accepted = g.accepted;
  A.guess_diag = g.diag;
  A.guess_sweeps = g.x ? g.sweeps : 0;
  A.guess_omega = g.omega;
  A.want_tangent = want_tangent ? 1 : 0;
  A.split_factor = (want_tangent && split_local_factor(c)) ? 1 : 0;
  A.phase = D.prof ? D.phase : nullptr;
  A.reuse = (D.local_reuse_active && D.local_factors_valid) ? 1 : 0;
  CK(cudaMemsetAsync(D.ov.queue, 0, sizeof(int32_t), D.s));
  dispatch_local_newton(c, c.ov, A, local_threads(c));
  if (A.split_factor) {
    if (fp32_local(c)) LAUNCH(D, k_local_factor<float>, c.ov.count, 256, factor_plan<float>(c.ov.max_b).total, A);
    else LAUNCH(D, k_local_factor<double>, c.ov.count, 256, factor_plan<double>(c.ov.max_b).total, A);
  }
}

void launch_local_apply(Context& c, const double* v, const double* add, double* out) {
  Dev& D = *c.dev;
  LocalArgs A = make_args(c, c.ov, D.ov);
  A.v = v;
  A.add = add;
  A.out = out;
  // the solves need warp 0 plus one thread per coupled row (32 + b); small CTAs let more
  // subdomains be in flight on every SM, which is what hides the latency of the solves
  const int T = apply_threads(c);
  if (fp32_local(c)) {
    const size_t sm = apply_plan<float>(c.ov.max_n, c.ov.max_nt).total;
    LAUNCH(D, k_local_apply<float>, c.ov.count, T, sm, A);
  } else {
    const size_t sm = apply_plan<double>(c.ov.max_n, c.ov.max_nt).total;
    LAUNCH(D, k_local_apply<double>, c.ov.count, T, sm, A);
  }
}

// ---- autotuner (nls_options.autotune) -------------------------------------------------------
// Candidates are timed with CUDA events on the context's own data and the fastest is kept for
// the life of the context.  Every candidate computes the same quantities (only the order of
// the reductions inside a subdomain differs), so the timed launches double as warm-up.
template <typename F>
float time_on_stream(Dev& D, F&& f) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, D.s));
  f();
  CK(cudaEventRecord(b, D.s));
  CK(cudaEventSynchronize(b));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

void tune_local_newton(Context& c, const double* x, double* out, double load, const GuessProposal& guess) {
  Dev& D = *c.dev;
  if (D.newton_tuned || !c.opt.autotune || c.opt.threads_per_block) return;
  const int need = min_local_threads(c);
  const int cand[2] = {128, 256};
  // warm-up with the fixed choice (first touch of the factor storage and the caches)
  launch_local_newton(c, x, out, load, guess, true);
  double best = INFINITY;
  int bestT = 0;
  for (int i = 0; i < 2; ++i) {
    if (cand[i] < need) continue;
    D.newton_T = cand[i];
    const float ms = time_on_stream(D, [&] { launch_local_newton(c, x, out, load, guess, true); });
    D.newton_ms[i] = ms;
    if (ms < best) {
      best = ms;
      bestT = cand[i];
    }
  }
  D.newton_T = bestT;
  D.newton_tuned = true;
}

void tune_local_apply(Context& c, const double* v, double* out) {
  Dev& D = *c.dev;
  if (D.apply_tuned || !c.opt.autotune) return;
  const int need = std::max(64, min_local_threads(c));
  std::vector<int> cand;
  for (int T : {need, need + 32, need + 64, 128, 192, 256})
    if (T >= need && T <= 256 && std::find(cand.begin(), cand.end(), T) == cand.end()) cand.push_back(T);
  D.apply_T = need;
  launch_local_apply(c, v, nullptr, out);  // warm-up
  double best = INFINITY;
  int bestT = need;
  for (int T : cand) {
    D.apply_T = T;
    float ms = INFINITY;
    for (int rep = 0; rep < 2; ++rep)
      ms = std::min(ms, time_on_stream(D, [&] { launch_local_apply(c, v, nullptr, out); }));
    if (ms < best) {
      best = ms;
      bestT = T;
    }
  }
  D.apply_T = bestT;
  D.apply_tuned = true;
}

// ---- coarse ---------------------------------------------------------------------------------
LocalArgs coarse_args(Context& c) {
  Dev& D = *c.dev;
  LocalArgs A = make_args(c, c.nov, D.nov);
  A.phi = D.phi;
  A.phi_off = D.phi_off;
  A.cj_ptr = D.cj_ptr;
  A.Y = D.Y;
  A.blk = D.blk;
  A.blk_off = D.blk_off;
  return A;
}

size_t coarse_factor_smem(const Context& c, bool f32) {
  const size_t fs = f32 ? sizeof(float) : sizeof(double);
  const size_t BS = f32 ? dev::SolveBlock<float>::BS : dev::SolveBlock<double>::BS;
  const size_t R = (size_t)dev::band_lu_window_rows(c.cs.b0);
  return fs * (R * dev::band_lu_window_stride(c.cs.b0) + R + 4 * BS * (BS + 1)) + 16;
}

// A_0(x) = P_0^T DF(x) P_0 -> band -> factor.  Returns false on a bad pivot.
void coarse_matrix_launch(Context& c, const double* x);
void coarse_inverse_launch(Context& c);

// Reads the coarse factorization's status word (synchronises the stream).
bool coarse_status_ok(Dev& D) {
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, D.cstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, D.s));
  sync(D);
  if (st == ST_TIMEOUT) throw DeviceTimeout("a tile of the coarse factorization gave up waiting for its operands");
  return st == ST_OK;
}
// The same, after checking that no coarse cluster solve gave up waiting.
bool coarse_status_ok(Context& c) {
  tlu_check_solves(c);
  return coarse_status_ok(*c.dev);
}

bool coarse_matrix(Context& c, const double* x) {
  coarse_matrix_launch(c, x);
  return coarse_status_ok(c);
}

// A_0(x) = P_0^T DF(x) P_0 in band storage (D.A0): Galerkin blocks per non-overlapping subdomain
// and their gather.
void coarse_assemble_launch(Context& c, const double* x) {
  Dev& D = *c.dev;
  LocalArgs A = coarse_args(c);
  A.x = x;
  const int T = 256;
  const size_t sm = smem_plan<double>(c.nov.max_n, c.nov.max_nt, c.nov.max_b, false).total;
  if (c.law == NLS_LAW_DIFFUSION) LAUNCH(D, (k_galerkin<NLS_LAW_DIFFUSION>), c.nov.count, T, sm, A);
  else LAUNCH(D, (k_galerkin<NLS_LAW_NEOHOOKE>), c.nov.count, T, sm, A);
  const int64_t ne = (int64_t)c.cs.N0 * (2 * c.cs.b0 + 1);
  LAUNCH(D, k_a0_gather, grid_for(ne), 256, 0, ne, D.a0_ptr, D.a0_src, D.blk, D.A0);
}

// Band factorization of D.A0 (one CTA; its size autotuned at the first call) into the packed
// solve operands; the status word is read by coarse_status_ok.
void coarse_factor_launch(Context& c) {
  Dev& D = *c.dev;
  if (D.tlu) {
    tlu_factor(c);
    return;
  }
  const bool f32 = fp32_coarse(c);
  const size_t fsm = coarse_factor_smem(c, f32);
  auto factor = [&](int T) {
    if (f32)
      LAUNCH(D, k_coarse_factor<float>, 1, T, fsm, c.cs.N0, c.cs.b0, D.A0, (float*)D.A0f, (float*)D.A0dinv,
             D.cstatus);
    else
      LAUNCH(D, k_coarse_factor<double>, 1, T, fsm, c.cs.N0, c.cs.b0, D.A0, (double*)D.A0f, (double*)D.A0dinv,
             D.cstatus);
  };
  if (c.opt.autotune && !D.coarse_tuned) {
    // the factorization reads A_0 and overwrites its own outputs: every candidate is a full,
    // valid factorization; the fastest CTA size is kept
    double best = INFINITY;
    int bestT = 1024;
    for (int T : {256, 512, 1024}) {
      const float ms = time_on_stream(D, [&] { factor(T); });
      if (ms < best) {
        best = ms;
        bestT = T;
      }
    }
    D.coarse_T = bestT;
    D.coarse_tuned = true;
  }
  factor(D.coarse_T);
}

void coarse_matrix_launch(Context& c, const double* x) {
  coarse_assemble_launch(c, x);
  coarse_factor_launch(c);
}

void coarse_solve(Context& c, const double* g, double* z) {
  Dev& D = *c.dev;
  if (D.ainv_valid) {
    // z = A_0^-1 g, then (FP32 inverse) up to min(ir_max_sweeps, 3) refinement steps
    // z += A_0^-1 (g - A_0 z) until ||g - A_0 z|| <= ir_rtol ||g||: a fixed sequence of launches
    // (graph-capturable) whose steps after convergence return at once
    const int N0 = c.cs.N0;
    const dim3 gg((N0 + 31) / 32, kGemvChunks);
    const bool f32 = fp32_coarse(c);
    auto apply_inverse = [&](const double* rhs, int accumulate, const int* skip, int* reset) {
      if (f32) LAUNCH(D, k_dense_gemv_t<float>, gg, 256, 0, N0, (const float*)D.ainv, rhs, D.gpart, skip);
      else LAUNCH(D, k_dense_gemv_t<double>, gg, 256, 0, N0, (const double*)D.ainv, rhs, D.gpart, skip);
      LAUNCH(D, k_gemv_finish, grid_for(N0), 256, 0, N0, kGemvChunks, D.gpart, z, accumulate, skip, reset);
    };
    apply_inverse(g, 0, nullptr, D.cflag);
    const int sweeps = f32 ? std::min(c.opt.ir_max_sweeps, 3) : 0;
    for (int sw = 0; sw < sweeps; ++sw) {
      LAUNCH(D, k_coarse_residual, (N0 + 7) / 8, 256, 0, N0, c.cs.b0, D.A0, g, z, D.cres, D.cpart,
             (unsigned*)(D.cflag + 1), D.cflag, c.opt.ir_rtol);
      apply_inverse(D.cres, 1, D.cflag, nullptr);
    }
    return;
  }
  // band factors: one solve in one CTA, then (FP32 factors) up to ir_max_sweeps refinement steps
  // z += A_0^-1 (g - A_0 z) with the FP64 residual on every SM; the same fixed launch sequence
  // as above, the steps after convergence returning at once
  const int N0 = c.cs.N0;
  const bool f32 = fp32_coarse(c);
  const int T = coarse_solve_threads(c);
  auto band_solve = [&](const double* rhs, int accumulate, const int* skip, int* reset) {
    if (tlu_solve(c, rhs, z, accumulate, skip, reset)) return;  // tiled factors: the cluster solve
    if (f32)
      LAUNCH(D, k_coarse_band_solve<float>, 1, T, sizeof(float) * N0, N0, c.cs.b0, (const float*)D.A0dinv, rhs, z,
             accumulate, skip, reset, c.opt.l2_prefetch);
    else
      LAUNCH(D, k_coarse_band_solve<double>, 1, T, sizeof(double) * N0, N0, c.cs.b0, (const double*)D.A0dinv, rhs, z,
             accumulate, skip, reset, c.opt.l2_prefetch);
  };
  band_solve(g, 0, nullptr, D.cflag);
  const int sweeps = f32 ? c.opt.ir_max_sweeps : 0;
  for (int sw = 0; sw < sweeps; ++sw) {
    LAUNCH(D, k_coarse_residual, (N0 + 7) / 8, 256, 0, N0, c.cs.b0, D.A0, g, z, D.cres, D.cpart,
           (unsigned*)(D.cflag + 1), D.cflag, c.opt.ir_rtol);
    band_solve(D.cres, 1, D.cflag, nullptr);
  }
}

// x = u - P0 c
void p0_update(Context& c, const double* u, const double* cv, double* x) {
  Dev& D = *c.dev;
  LAUNCH(D, k_p0_apply, grid_for(c.N), 256, 0, c.N, D.p0_rowptr, D.p0_col, D.p0_val, cv, 1.0, u, -1.0, x);
}

void p0t(Context& c, const double* v, double* g) {
  Dev& D = *c.dev;
  LAUNCH(D, k_p0t_apply, c.cs.N0, 256, 0, c.cs.N0, D.p0t_rowptr, D.p0t_col, D.p0t_val, v, g);
}

struct CoarseResult {
  int its = 0;
  int status = ST_OK;
};

// Coarse Newton for Eq. 9: g(c) = P0^T F(u - P0 c) = 0, c <- c + alpha A0^-1 g.  Leaves
// D.c = T_0(u) and D.u0 = u - P0 T_0(u).
CoarseResult coarse_newton(Context& c, const double* u, double load) {
  Dev& D = *c.dev;
  CoarseResult R;
  const int N0 = c.cs.N0;
  CK(cudaMemsetAsync(D.c, 0, sizeof(double) * N0, D.s));
  CK(cudaMemcpyAsync(D.u0, u, sizeof(double) * c.N, cudaMemcpyDeviceToDevice, D.s));
  global_residual(c, D.u0, D.F, load);
  p0t(c, D.F, D.g);
  double gn = norm2(D, N0, D.g);
  if (!std::isfinite(gn)) {
    R.status = ST_NONFINITE;
    return R;
  }
  const double tol = std::max(c.opt.inner_atol, c.opt.inner_rtol * gn);
  // With coarse_reuse the iteration starts from the factorization of the previous tangent
  // phase's A_0 (chord steps, solved with its explicit inverse) and forms A_0 at the current
  // point only when a step contracts ||g|| by less than half or fails the line search; the
  // stopping test is the same either way.
  bool refresh = !(c.opt.coarse_reuse && D.coarse_fact_valid);
  while (gn > tol) {
    if (R.its >= c.opt.inner_maxit) {
      R.status = ST_MAXIT;
      break;
    }
    const bool chord = !refresh;
    if (!chord) {
      D.ainv_valid = false;  // the explicit inverse belongs to an older A_0
      D.coarse_fact_valid = coarse_matrix(c, D.u0);
      if (!D.coarse_fact_valid) {
        R.status = ST_PIVOT;
        break;
      }
      // the explicit inverse costs about a third of one band solve, and every solve with it
      // (GEMV + FP64 refinement) a tenth
      if (D.ainv) {
        coarse_inverse_launch(c);
        D.ainv_valid = true;
      }
    }
    coarse_solve(c, D.g, D.dc);
    double alpha = 1.0, gtn = INFINITY;
    bool accepted = false;
    for (int trial = 0; trial < c.opt.ls_trials; ++trial) {
      LAUNCH(D, k_axpby, grid_for(N0), 256, 0, (int64_t)N0, 1.0, D.c, alpha, D.dc, D.ct);
      p0_update(c, u, D.ct, D.x);
      global_residual(c, D.x, D.F, load);
      p0t(c, D.F, D.gt);
      gtn = norm2(D, N0, D.gt);
      if (std::isfinite(gtn) && gtn <= (1.0 - c.opt.armijo * alpha) * gn) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
    }
    if (!accepted && chord) {
      refresh = true;  // retry the step with A_0 at the current point
      continue;
    }
    R.its += 1;
    if (!accepted) {
      R.status = ST_LS;
      break;
    }
    refresh = !c.opt.coarse_reuse || gtn > 0.5 * gn;
    std::swap(D.c, D.ct);
    std::swap(D.u0, D.x);
    std::swap(D.g, D.gt);
    gn = gtn;
  }
  return R;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// setup on the device
// ------------------------------------------------------------------------------------------
namespace {

void upload_set(Dev& D, const LocalSet& h, DeviceLocalSet& d, bool fp32_factor, bool with_dinv = true) {
  d.count = h.count;
  d.meta = D.upload(h.meta);
  d.tnode_gid = D.upload(h.tnode_gid);
  d.elem_gid = D.upload(h.elem_gid);
  d.lconn = D.upload(h.lconn);
  d.color_ptr = D.upload(h.color_ptr);
  d.rowptr = D.upload(h.rowptr);
  d.colidx = D.upload(h.colidx);
  d.epos = D.upload(h.epos);
  d.owned = D.upload(h.owned);
  d.csr_val = D.alloc<double>(h.total_nnz);
  if (fp32_factor) {
    d.factor = D.alloc<float>(h.total_factor);
    if (with_dinv) d.dinv = D.alloc<float>(h.total_dinv);
  } else {
    d.factor = D.alloc<double>(h.total_factor);
    if (with_dinv) d.dinv = D.alloc<double>(h.total_dinv);
  }
  d.w = D.alloc<double>(h.total_n);
  d.work = D.alloc<double>(3 * (size_t)h.total_n);
  d.its = D.alloc<int32_t>(h.count);
  d.chord = D.alloc<int32_t>(h.count);
  d.status = D.alloc<int32_t>(h.count);
  // longest first: cost ~ n b^2
  std::vector<int32_t> order(h.count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double ca = (double)h.meta[a].n * h.meta[a].b * h.meta[a].b, cb = (double)h.meta[b].n * h.meta[b].b * h.meta[b].b;
    return ca > cb;
  });
  d.order = D.upload(order);
  d.queue = D.alloc<int32_t>(1);
}

}  // namespace

// Energy-minimising extension of the interface values of the coarse basis (RGDSW, Section 2)
// with K = DF(u^(0)), u^(0) = Dirichlet data and zero elsewhere, then the values of P_0 and
// P_0^T.  The factors of the non-overlapping problems are needed for the extension only.
// RGDSW coarse basis: the interface values (host) extended into every non-overlapping
// subdomain by the energy-minimising (harmonic) extension with DF(x) (k_harmonic), then P_0 and
// P_0^T gathered.  x = nullptr: the Dirichlet data u^(0) (the basis built once, at setup);
// otherwise the current outer iterate (coarse_rebuild).
void coarse_extension(Context& c, const double* x = nullptr) {
  Dev& D = *c.dev;
  Coarse& cs = c.cs;
  const int64_t N = c.N;
  const size_t lim = D.smem_optin;
  auto need = [&](size_t b, const char* what) {
    if (b > lim) throw std::runtime_error(std::string(what) + " needs more shared memory than the device offers");
  };
  if (!D.nov.factor) D.nov.factor = D.alloc<double>(c.nov.total_factor);
  CK(cudaMemcpyAsync(D.phi, cs.phi_host.data(), sizeof(double) * cs.phi_host.size(), cudaMemcpyHostToDevice, D.s));
  CK(cudaMemcpyAsync(D.x, x ? x : D.ubc, sizeof(double) * N, cudaMemcpyDeviceToDevice, D.s));
  LocalArgs A = coarse_args(c);
  A.x = D.x;
  const size_t sm = harmonic_plan(c.nov.max_n, c.nov.max_nt, c.nov.max_b).total;
  need(sm, "coarse harmonic extension");
  if (c.law == NLS_LAW_DIFFUSION) LAUNCH(D, k_harmonic<NLS_LAW_DIFFUSION>, c.nov.count, 256, sm, A);
  else LAUNCH(D, k_harmonic<NLS_LAW_NEOHOOKE>, c.nov.count, 256, sm, A);
  std::vector<int32_t> st(c.nov.count);
  CK(cudaMemcpyAsync(st.data(), D.nov.status, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost, D.s));
  sync(D);
  for (int32_t s : st)
    if (s != ST_OK) throw std::runtime_error("coarse harmonic extension hit a zero pivot");
  const int64_t np = (int64_t)cs.p0_col.size();
  LAUNCH(D, k_gather_values, grid_for(np), 256, 0, np, D.p0_src, D.phi, D.p0_val);
  LAUNCH(D, k_gather_values32, grid_for(np), 256, 0, np, D.p0t_src, D.p0_val, D.p0t_val);
  if (!c.opt.coarse_rebuild) {  // rebuilt every outer iteration otherwise: keep the factor storage
    D.release(D.nov.factor);
    D.nov.factor = nullptr;
  }
}

int device_setup(Context& c) {
  try {
    CK(cudaSetDevice(c.device));
    Dev* Dp = new Dev();
    c.dev = Dp;
    Dev& D = *Dp;
    // NULL selects the legacy default stream, which orders against every blocking stream of
    // the caller (a torch tensor filled on the default stream is complete before we read it).
    D.s = (cudaStream_t)c.stream;
    c.own_stream = false;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, c.device));
    D.nsm = prop.multiProcessorCount;
    D.smem_optin = prop.sharedMemPerBlockOptin;
    D.conn = D.upload(c.conn);
    D.geom = D.upload(c.geom);
    std::vector<double> k = c.k_elem;
    if (k.empty()) k.assign(c.n_elems, 1.0);
    D.kcoef = D.upload(k);
    D.fext = D.upload(c.fext);
    D.ubc = D.upload(c.ubc);
    D.free_dof = D.upload(c.free_dof);
    D.g_elem = D.upload(c.g_elem);
    {
      // node stars as element-local references (e nen + a), ascending element ids
      std::vector<int32_t> ref(c.star_el.size());
      for (int64_t v = 0; v < c.n_nodes; ++v)
        for (int64_t k = c.star_ptr[v]; k < c.star_ptr[v + 1]; ++k) {
          const int32_t e = c.star_el[k];
          int a = 0;
          while (a < c.nen - 1 && c.conn[(int64_t)e * c.nen + a] != v) ++a;
          ref[k] = e * c.nen + a;
        }
      D.star_ptr = D.upload(c.star_ptr);
      D.star_ref = D.upload(ref);
      D.Re = D.alloc<double>((size_t)c.n_elems * c.nen * c.ndof);
    }
    D.g_rowptr = D.upload(c.g_rowptr);
    D.g_col = D.upload(c.g_col);
    D.g_epos = D.upload(c.g_epos);
    D.g_val = D.alloc<double>(c.g_col.size());
    upload_set(D, c.ov, D.ov, fp32_local(c));
    const int N = (int)c.N;
    D.u = D.alloc<double>(N);
    D.ut = D.alloc<double>(N);
    D.x = D.alloc<double>(N);
    D.u0 = D.alloc<double>(N);
    D.Fx = D.alloc<double>(N);
    D.F = D.alloc<double>(N);
    D.t1 = D.alloc<double>(N);
    D.t2 = D.alloc<double>(N);
    D.w0 = D.alloc<double>(N);
    D.gx = D.alloc<double>(N);
    D.m = std::max(1, std::min(c.opt.gmres_restart, kMaxGmresVecs / 2 - 2));
    D.V = D.alloc<double>((size_t)(D.m + 1) * N);
    CK(cudaMemsetAsync(D.V, 0, sizeof(double) * (size_t)(D.m + 1) * N, D.s));
    D.partial = D.alloc<double>((size_t)kVecWarps * (kMaxGmresVecs + 2));
    D.scal = D.alloc<double>(kMaxGmresVecs + 8);
    D.coef = D.alloc<double>(kMaxGmresVecs + 8);
    D.gR = D.alloc<double>((size_t)D.m * D.m);
    D.gcs = D.alloc<double>(D.m);
    D.gsn = D.alloc<double>(D.m);
    D.gg = D.alloc<double>(D.m + 1);
    D.gst = (GmresState*)D.alloc<double>(4);
    D.bad = D.alloc<int>(4);
    D.phase = D.alloc<unsigned long long>(8);
    CK(cudaMemsetAsync(D.phase, 0, sizeof(unsigned long long) * 8, D.s));
    CK(cudaDeviceGetAttribute(&D.clock_khz, cudaDevAttrClockRate, c.device));
    CK(cudaMallocHost(&D.h_scal, sizeof(double) * (kMaxGmresVecs + 8)));
    // kernel attributes for large dynamic shared memory
    const size_t lim = D.smem_optin;
    auto need = [&](size_t b, const char* what) {
      if (b > lim) throw std::runtime_error(std::string(what) + " needs more shared memory than the device offers");
    };
    if (c.ov.max_b > 128)
      throw std::runtime_error("a local band matrix has a half bandwidth above 128 (" + std::to_string(c.ov.max_b) +
                               "); the local band factorisation supports 128");
    if (c.coarse_kind == NLS_COARSE_RGDSW && !coarse_tiles(c) && c.cs.b0 > kMaxBandB0)
      throw std::runtime_error("the coarse matrix has a half bandwidth of " + std::to_string(c.cs.b0) +
                               "; the one-CTA band factorisation supports " + std::to_string(kMaxBandB0) +
                               " (the tiled one, coarse_factor = NLS_COARSE_FACTOR_TILES, up to " +
                               std::to_string(kMaxSolveB0) + ")");
    if (c.coarse_kind == NLS_COARSE_RGDSW && c.cs.b0 > kMaxSolveB0)
      throw std::runtime_error("the coarse matrix has a half bandwidth of " + std::to_string(c.cs.b0) +
                               "; the coarse solves support " + std::to_string(kMaxSolveB0));
    need(local_newton_smem<float>(c.ov), "local Newton (FP32 factors)");
    if (!fp32_local(c)) need(local_newton_smem<double>(c.ov), "local Newton (FP64 factors)");
    set_smem(k_local_newton<NLS_LAW_DIFFUSION, float, 128>, lim);
    set_smem(k_local_newton<NLS_LAW_DIFFUSION, double, 128>, lim);
    set_smem(k_local_newton<NLS_LAW_NEOHOOKE, float, 128>, lim);
    set_smem(k_local_newton<NLS_LAW_NEOHOOKE, double, 128>, lim);
    set_smem(k_local_newton<NLS_LAW_DIFFUSION, float, 256>, lim);
    set_smem(k_local_newton<NLS_LAW_DIFFUSION, double, 256>, lim);
    set_smem(k_local_newton<NLS_LAW_NEOHOOKE, float, 256>, lim);
    set_smem(k_local_newton<NLS_LAW_NEOHOOKE, double, 256>, lim);
    set_smem(k_local_apply<float>, lim);
    set_smem(k_local_factor<float>, lim);
    set_smem(k_local_factor<double>, lim);
    set_smem(k_guess_smooth<NLS_LAW_DIFFUSION>, lim);
    set_smem(k_guess_smooth<NLS_LAW_NEOHOOKE>, lim);
    set_smem(k_local_apply<double>, lim);
    set_smem(k_harmonic<NLS_LAW_DIFFUSION>, lim);
    set_smem(k_harmonic<NLS_LAW_NEOHOOKE>, lim);
    set_smem(k_galerkin<NLS_LAW_DIFFUSION>, lim);
    set_smem(k_galerkin<NLS_LAW_NEOHOOKE>, lim);
    set_smem(k_coarse_factor<float>, lim);
    set_smem(k_coarse_factor<double>, lim);
    if (c.coarse_kind == NLS_COARSE_RGDSW) {
      Coarse& cs = c.cs;
      if (cs.N0 == 0) throw std::runtime_error("the partition has no coarse nodes (one subdomain?)");
      if (!coarse_tiles(c)) need(coarse_factor_smem(c, fp32_coarse(c)), "coarse band factorization");
      need((fp32_coarse(c) ? sizeof(float) : sizeof(double)) * (size_t)cs.N0, "coarse band solve");
      upload_set(D, c.nov, D.nov, false, false);
      D.phi = D.upload(cs.phi_host);
      D.phi_off = D.upload(cs.phi_off);
      D.cj_ptr = D.upload(cs.cj_ptr);
      D.Y = D.alloc<double>(cs.phi_total);
      D.blk = D.alloc<double>(cs.blk_total);
      D.blk_off = D.upload(cs.blk_off);
      D.a0_ptr = D.upload(cs.a0_ptr);
      D.a0_src = D.upload(cs.a0_src);
      D.A0 = D.alloc<double>((size_t)cs.N0 * (2 * cs.b0 + 1));
      const size_t ndinv = (size_t)packed_solve_entries(cs.N0, cs.b0);
      if (fp32_coarse(c)) {
        D.A0f = D.alloc<float>((size_t)cs.N0 * (2 * cs.b0 + 1));
        D.A0dinv = D.alloc<float>(ndinv);
      } else {
        D.A0f = D.alloc<double>((size_t)cs.N0 * (2 * cs.b0 + 1));
        D.A0dinv = D.alloc<double>(ndinv);
      }
      D.cstatus = D.alloc<int32_t>(1);
      // refinement of the coarse solves: per-CTA partial norms, converged flag and ticket counter
      D.cpart = D.alloc<double>(2 * (size_t)((cs.N0 + 7) / 8));
      D.cflag = D.alloc<int>(2);
      CK(cudaMemsetAsync(D.cflag, 0, 2 * sizeof(int), D.s));
      set_smem(k_coarse_band_solve<float>, lim);
      set_smem(k_coarse_band_solve<double>, lim);
      if (coarse_tiles(c)) tlu_prepare(c, fp32_coarse(c));
      if (cs.N0 <= kMaxInverseN0) {
        if (fp32_coarse(c)) D.ainv = D.alloc<float>((size_t)cs.N0 * cs.N0);
        else D.ainv = D.alloc<double>((size_t)cs.N0 * cs.N0);
        D.gpart = D.alloc<double>((size_t)cs.N0 * kGemvChunks);
        set_smem(k_coarse_inverse<float>, lim);
        set_smem(k_coarse_inverse<double>, lim);
      }
      D.p0_rowptr = D.upload(cs.p0_rowptr);
      D.p0_col = D.upload(cs.p0_col);
      D.p0_src = D.upload(cs.p0_src);
      D.p0_val = D.alloc<double>(cs.p0_col.size());
      D.p0t_rowptr = D.upload(cs.p0t_rowptr);
      D.p0t_col = D.upload(cs.p0t_col);
      D.p0t_src = D.upload(cs.p0t_src);
      D.p0t_val = D.alloc<double>(cs.p0t_col.size());
      D.c = D.alloc<double>(cs.N0);
      D.ct = D.alloc<double>(cs.N0);
      D.dc = D.alloc<double>(cs.N0);
      D.g = D.alloc<double>(cs.N0);
      D.gt = D.alloc<double>(cs.N0);
      D.tg = D.alloc<double>(cs.N0);  // the tangent's coarse right-hand side (never swapped)
      D.cres = D.alloc<double>(cs.N0);
      coarse_extension(c);
    }
    sync(D);
    c.device_bytes = D.bytes;
  } catch (const DeviceTimeout& ex) {
    c.last_error = ex.what();
    return NLS_E_DEVICE_TIMEOUT;
  } catch (const CudaFailure& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  } catch (const std::bad_alloc&) {
    c.last_error = "host allocation failed";
    return NLS_E_NOMEM;
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_ARG;
  }
  return NLS_OK;
}

int device_set_coefficients(Context& c) {
  try {
    Dev& D = *c.dev;
    CK(cudaSetDevice(c.device));
    std::vector<double> k = c.k_elem;
    if (k.empty()) k.assign(c.n_elems, 1.0);
    CK(cudaMemcpyAsync(D.kcoef, k.data(), sizeof(double) * k.size(), cudaMemcpyHostToDevice, D.s));
    CK(cudaMemcpyAsync(D.fext, c.fext.data(), sizeof(double) * c.fext.size(), cudaMemcpyHostToDevice, D.s));
    if (c.coarse_kind == NLS_COARSE_RGDSW) coarse_extension(c);
    D.coarse_fact_valid = false;
    D.ainv_valid = false;
    D.tangent_ready = false;
    guess_coefficients_changed(c);
    sync(D);
  } catch (const CudaFailure& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_ARG;
  }
  return NLS_OK;
}

int device_upload_fext(Context& c) {
  try {
    Dev& D = *c.dev;
    CK(cudaSetDevice(c.device));
    CK(cudaMemcpyAsync(D.fext, c.fext.data(), sizeof(double) * c.fext.size(), cudaMemcpyHostToDevice, D.s));
    sync(D);
  } catch (const CudaFailure& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

void device_free(Context& c) {
  if (!c.dev) return;
  Dev& D = *c.dev;
  cudaSetDevice(c.device);
  if (D.s) cudaStreamSynchronize(D.s);
  guess_free(c);
  tlu_free(c);
  D.reset_graphs();
  if (D.cap) cudaStreamDestroy(D.cap);
  if (D.s2) cudaStreamSynchronize(D.s2), cudaStreamDestroy(D.s2);
  if (D.ev_u0) cudaEventDestroy(D.ev_u0);
  if (D.ev_coarse) cudaEventDestroy(D.ev_coarse);
  for (void* p : D.allocs)
    if (p) cudaFree(p);
  if (D.h_scal) cudaFreeHost(D.h_scal);
  for (auto& r : D.evs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (c.own_stream && D.s) cudaStreamDestroy(D.s);
  c.own_stream = false;
  delete c.dev;
  c.dev = nullptr;
}

// ------------------------------------------------------------------------------------------
// F_x, tangent, GMRES, outer Newton
// ------------------------------------------------------------------------------------------
namespace {

struct FxInfo {
  int coarse_its = 0;
  int coarse_status = ST_OK;
  int64_t local_its = 0;
  int64_t local_chord = 0;
  int local_failures = 0;
  int first_failed = -1;
  bool pivot_failure = false;
};

// Explicit A_0^-1 from the current coarse factors (N0 <= kMaxInverseN0), issued on D.s; coarse solves use
// it (refined in FP64 against A_0 where it is applied) once ainv_valid is set.
void coarse_inverse_launch(Context& c) {
  Dev& D = *c.dev;
  if (!D.ainv) return;
  const int N0 = c.cs.N0;
  const int T = std::max(64, (32 + c.cs.b0 + 31) / 32 * 32);
  const int grid = std::min(N0, D.nsm * 8);
  if (fp32_coarse(c))
    LAUNCH(D, k_coarse_inverse<float>, grid, T, sizeof(float) * N0, N0, c.cs.b0, (const float*)D.A0dinv,
           (float*)D.ainv, c.opt.l2_prefetch);
  else
    LAUNCH(D, k_coarse_inverse<double>, grid, T, sizeof(double) * N0, N0, c.cs.b0, (const double*)D.A0dinv,
           (double*)D.ainv, c.opt.l2_prefetch);
}

// The tangent phase's coarse work at u_0, first part (issued on D.s): DF(u_0) for the coarse term
// of Eq. 12 and A_0(u_0).  These kernels use many CTAs and run before the persistent local
// Newton launch, which then holds every SM.
void tangent_coarse_assemble(Context& c) {
  Dev& D = *c.dev;
  global_jacobian(c, D.u0);
  D.ainv_valid = false;
  coarse_assemble_launch(c, D.u0);
}

// Second part (issued on the high-priority second stream): the one-CTA factorization of A_0(u_0),
// placed beside the local Newton CTAs, and (N_0 <= kMaxInverseN0) the explicit inverse the GMRES
// iterations' coarse solves use.  The factorization's status is read by the caller.
void tangent_coarse_factor(Context& c) {
  coarse_factor_launch(c);
  coarse_inverse_launch(c);
}

// F_x(u) into D.Fx; prepares everything the tangent needs.
FxInfo evaluate_Fx(Context& c, const double* u, double load, double* t_inner, double* t_coarse) {
  Dev& D = *c.dev;
  FxInfo info;
  const int cp = c.opt.coupling;
  CK(cudaMemsetAsync(D.Fx, 0, sizeof(double) * c.N, D.s));
  auto t0 = std::chrono::steady_clock::now();
  const double* point = u;
  if (cp != NLS_COUPLING_ONE) {
    CoarseResult cr = coarse_newton(c, u, load);
    info.coarse_its = cr.its;
    info.coarse_status = cr.status;
    if (cp == NLS_COUPLING_HYBRID) point = D.u0;
  }
  sync(D);
  auto t1 = std::chrono::steady_clock::now();
  // The tangent phase's coarse work depends on u_0 only: it goes on a second stream of the
  // highest priority, issued before the batched local solves, so that it runs beside them.  The
  // persistent local Newton grid fills every SM, so how it shares them depends on its occupancy:
  // - several CTAs per SM: DF(u_0) and A_0(u_0) (many CTAs) go first on this stream, and the
  //   single-CTA factorization of A_0 is dispatched together with the local solves, beside
  //   some of their CTAs (the kernel pulls subdomains from a work counter, so a CTA of it that
  //   starts late only takes fewer of them);
  // - one CTA per SM (none can share an SM with the factorization): the whole chain goes on
  //   the second stream, its assembly overlapping the start of the local solves, and the local
  //   Newton grid leaves one SM to the factorization.
  // The tiled factorization spreads every step over many CTAs: it cannot live in the corner of the
  // machine the local grid leaves, so it runs alone on the main stream, before the local solves.
  const bool two_level = cp != NLS_COUPLING_ONE;
  const bool serial_coarse = two_level && D.tlu != nullptr;
  const bool spare_sm = two_level && !serial_coarse && newton_ctas_per_sm(c) == 1;
  if (serial_coarse) {
    tangent_coarse_assemble(c);
    tangent_coarse_factor(c);
  } else if (two_level) {
    if (!spare_sm) tangent_coarse_assemble(c);
    if (!D.s2) {
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      CK(cudaStreamCreateWithPriority(&D.s2, cudaStreamNonBlocking, greatest));
      CK(cudaEventCreateWithFlags(&D.ev_u0, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&D.ev_coarse, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(D.ev_u0, D.s));
    CK(cudaStreamWaitEvent(D.s2, D.ev_u0, 0));
    std::swap(D.s, D.s2);
    try {
      if (spare_sm) tangent_coarse_assemble(c);
      tangent_coarse_factor(c);
    } catch (...) {
      std::swap(D.s, D.s2);
      throw;
    }
    CK(cudaEventRecord(D.ev_coarse, D.s));
    std::swap(D.s, D.s2);
  }
  const GuessProposal proposal = guess_propose(c, point, load);
  tune_local_newton(c, point, D.Fx, load, proposal);
  D.coarse_beside = spare_sm;
  launch_local_newton(c, point, D.Fx, load, proposal, true);
  D.coarse_beside = false;
  D.local_factors_valid = true;  // every subdomain with status OK now holds its tangent factors
  guess_after_local(c, point, load, proposal.x != nullptr);
  std::vector<int32_t> its(c.ov.count), st(c.ov.count), ch(c.ov.count);
  CK(cudaMemcpyAsync(its.data(), D.ov.its, sizeof(int32_t) * its.size(), cudaMemcpyDeviceToHost, D.s));
  CK(cudaMemcpyAsync(st.data(), D.ov.status, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost, D.s));
  CK(cudaMemcpyAsync(ch.data(), D.ov.chord, sizeof(int32_t) * ch.size(), cudaMemcpyDeviceToHost, D.s));
  sync(D);
  auto t2 = std::chrono::steady_clock::now();
  for (int i = 0; i < c.ov.count; ++i) {
    info.local_its += its[i];
    info.local_chord += ch[i];
    if (st[i] != ST_OK) {
      info.local_failures += 1;
      if (info.first_failed < 0) info.first_failed = i;
      if (st[i] == ST_PIVOT) info.pivot_failure = true;
    }
  }
  if (two_level) {
    // F_x += P0 T_0(u); the coarse part of the tangent at u_0 = u - P0 T_0(u) comes from the
    // second stream
    LAUNCH(D, k_p0_apply, grid_for(c.N), 256, 0, c.N, D.p0_rowptr, D.p0_col, D.p0_val, D.c, 1.0, D.Fx, 1.0, D.Fx);
    if (!serial_coarse) CK(cudaStreamWaitEvent(D.s, D.ev_coarse, 0));
    D.coarse_fact_valid = coarse_status_ok(c);
    if (!D.coarse_fact_valid) info.pivot_failure = true;
    D.ainv_valid = D.coarse_fact_valid && D.ainv != nullptr;
  }
  sync(D);
  auto t3 = std::chrono::steady_clock::now();
  if (t_inner) *t_inner += std::chrono::duration<double>(t2 - t1).count();
  if (t_coarse) *t_coarse += std::chrono::duration<double>(t1 - t0).count() + std::chrono::duration<double>(t3 - t2).count();
  c.dev->tangent_ready = true;
  return info;
}

// y = DF_x v (Eq. 6 / Eq. 12)
void tangent(Context& c, const double* v, double* y) {
  Dev& D = *c.dev;
  const int cp = c.opt.coupling;
  if (cp == NLS_COUPLING_ONE) {
    launch_local_apply(c, v, nullptr, y);
    return;
  }
  // w0 = P0 A0^-1 P0^T DF(u0) v
  LAUNCH(D, k_spmv_free, grid_for(c.N), 256, 0, c.N, D.g_rowptr, D.g_col, D.g_val, D.free_dof, v, D.t1);
  p0t(c, D.t1, D.tg);
  coarse_solve(c, D.tg, D.dc);
  LAUNCH(D, k_p0_apply, grid_for(c.N), 256, 0, c.N, D.p0_rowptr, D.p0_col, D.p0_val, D.dc, 0.0, nullptr, 1.0, D.w0);
  if (cp == NLS_COUPLING_ADD) {
    launch_local_apply(c, v, D.w0, y);
  } else {
    LAUNCH(D, k_axpby, grid_for(c.N), 256, 0, c.N, 1.0, v, -1.0, D.w0, D.t2);
    launch_local_apply(c, D.t2, D.w0, y);
  }
}

struct GmresResult {
  int its = 0;
  double relres = 0.0;
  bool converged = false;
};

// GMRES(m), zero initial guess, classical Gram-Schmidt with one re-orthogonalisation (device
// multi-dots), Givens rotations and the least-squares update on the device.  Solution into D.gx.
//
// A cycle of up to m iterations runs without the host: with CUDA graphs it is one graph of m
// conditional (IF) nodes in a chain, node j holding iteration j's body (tangent application,
// two Gram-Schmidt passes, norm, scaling, Givens step); the Givens kernel of iteration j sets the
// shared condition to "continue" or "stop" (converged, breakdown, or the cycle's iteration limit),
// so no body after the last useful one is launched.  The host reads the cycle's state once, then
// the least-squares solve and the update run on the device.  The cycle graph holds device pointers
// and kernel arguments, so it is keyed by everything those depend on: the options, the
// coarse-solve form (explicit inverse or band factors), the tangent CTA size and the scratch
// vectors.  Without graphs (profiling, or cuda_graphs = 0) the same kernels run on the stream and
// the host reads the state after every iteration.
std::string cycle_graph_key(Context& c) {
  Dev& D = *c.dev;
  std::string key((const char*)&c.opt, sizeof(c.opt));
  key += D.ainv_valid ? 'i' : 'b';
  key += std::to_string(apply_threads(c)) + "," + std::to_string(D.m) + ",";
  // scratch vectors the tangent writes (some are swapped by the coarse Newton iteration)
  for (const void* p : {(const void*)D.t1, (const void*)D.t2, (const void*)D.w0, (const void*)D.tg,
                        (const void*)D.dc, (const void*)D.gpart, (const void*)D.cres,
                        (const void*)D.cpart, (const void*)D.cflag})
    key += std::to_string((uintptr_t)p) + ",";
  return key;
}

// Captures (first use) and launches the cycle graph; body(j, next, use) issues iteration j, whose
// Givens step sets `next` (the condition of node j + 1) when `use` is set.  The kernels of every
// body are counted apart, for the launch count once the cycle's length is known.
template <typename F>
void run_cycle_graph(Context& c, F&& body) {
  Dev& D = *c.dev;
  const std::string key = cycle_graph_key(c);
  if (key != D.graph_key || D.it_exec.empty()) {
    D.reset_graphs();
    D.graph_key = key;
    if (!D.cap) CK(cudaStreamCreateWithFlags(&D.cap, cudaStreamNonBlocking));
    cudaGraph_t G = nullptr;
    CK(cudaGraphCreate(&G, 0));
    const cudaStream_t saved = D.s;
    const int64_t l0 = D.launches;
    try {
      // one condition per node (a handle belongs to one conditional node): node 0 runs by default,
      // node j + 1 only when iteration j's Givens step sets its handle; all are reset at launch
      std::vector<cudaGraphConditionalHandle> h(D.m);
      for (int j = 0; j < D.m; ++j)
        CK(cudaGraphConditionalHandleCreate(&h[j], G, j == 0 ? 1u : 0u, cudaGraphCondAssignDefault));
      cudaGraphNode_t prev = nullptr;
      D.it_launches.assign(D.m, 0);
      for (int j = 0; j < D.m; ++j) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h[j];
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        CK(cudaGraphAddNode(&node, G, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &p));
        cudaGraph_t bg = p.conditional.phGraph_out[0];
        const int64_t lj = D.launches;
        CK(cudaStreamBeginCaptureToGraph(D.cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        D.s = D.cap;
        try {
          body(j, j + 1 < D.m ? h[j + 1] : cudaGraphConditionalHandle{}, j + 1 < D.m ? 1 : 0);
        } catch (...) {
          cudaGraph_t tmp = nullptr;
          cudaStreamEndCapture(D.cap, &tmp);
          throw;
        }
        D.s = saved;
        CK(cudaStreamEndCapture(D.cap, &bg));
        D.it_launches[j] = D.launches - lj;
        prev = node;
      }
      cudaGraphExec_t ex = nullptr;
      CK(cudaGraphInstantiate(&ex, G, 0));
      D.it_exec.assign(1, ex);
    } catch (...) {
      D.s = saved;
      D.launches = l0;
      cudaGraphDestroy(G);
      D.reset_graphs();
      throw;
    }
    cudaGraphDestroy(G);
    D.launches = l0;
  }
  CK(cudaGraphLaunch(D.it_exec[0], D.s));
}

GmresResult gmres(Context& c, const double* b) {
  Dev& D = *c.dev;
  const int64_t N = c.N;
  const int m = D.m;
  GmresResult R;
  tune_local_apply(c, b, D.t1);
  const bool graphs = c.opt.cuda_graphs && !D.prof;
  CK(cudaMemsetAsync(D.gx, 0, sizeof(double) * N, D.s));
  const double bn = norm2(D, N, b);
  if (bn == 0.0) {
    R.converged = true;
    return R;
  }
  double* r = D.t2;
  CK(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, D.s));
  double rn = bn;
  const double target = c.opt.gmres_rtol * bn;
  // iteration j of a cycle: w = DF_x v_j, CGS2 against v_0 .. v_j, h_{j+1,j} = ||w||, v_{j+1} =
  // w / h_{j+1,j}, Givens step (sets the graph condition when `use_handle`)
  auto body = [&](int j, cudaGraphConditionalHandle h, int use_handle) {
    double* vj = D.V + (size_t)j * N;
    double* w = D.V + (size_t)(j + 1) * N;
    tangent(c, vj, w);
    for (int pass = 0; pass < 2; ++pass) {
      LAUNCH(D, k_multidot_partial, kVecBlocks, kVecThreads, 0, N, j + 1, D.V, N, w, D.partial);
      LAUNCH(D, k_partial_final, std::min(j + 1, 64), 256, 0, j + 1, D.partial, D.scal + pass * (kMaxGmresVecs / 2));
      LAUNCH(D, k_multiaxpy, grid_for(N), 256, 0, N, j + 1, D.V, N, D.scal + pass * (kMaxGmresVecs / 2), -1.0, w);
    }
    LAUNCH(D, k_multidot_partial, kVecBlocks, kVecThreads, 0, N, 1, w, (int64_t)0, w, D.partial);
    LAUNCH(D, k_partial_final, 1, 256, 0, 1, D.partial, D.scal + kMaxGmresVecs);
    LAUNCH(D, k_sqrt_inplace, 1, 1, 0, D.scal + kMaxGmresVecs);
    LAUNCH(D, k_scale_inv, grid_for(N), 256, 0, N, w, D.scal + kMaxGmresVecs, w);
    LAUNCH(D, k_gmres_givens, 1, 32, 0, j, m, D.scal, D.gR, D.gcs, D.gsn, D.gg, D.gst, h, use_handle);
  };
  GmresState st;
  while (R.its < c.opt.gmres_maxit) {
    LAUNCH(D, k_axpby, grid_for(N), 256, 0, N, 1.0 / rn, r, 0.0, nullptr, D.V);
    const int limit = std::min(m, c.opt.gmres_maxit - R.its);
    LAUNCH(D, k_gmres_start, 1, 32, 0, m, rn, target, limit, D.gg, D.gst);
    if (graphs) {
      run_cycle_graph(c, body);
      CK(cudaMemcpyAsync(&st, D.gst, sizeof(st), cudaMemcpyDeviceToHost, D.s));
      sync(D);
      for (int j = 0; j < st.j; ++j) D.launches += D.it_launches[j];
    } else {
      for (int j = 0; j < limit; ++j) {
        body(j, cudaGraphConditionalHandle{}, 0);
        CK(cudaMemcpyAsync(&st, D.gst, sizeof(st), cudaMemcpyDeviceToHost, D.s));
        sync(D);
        if (st.done || st.j >= limit) break;
      }
    }
    // y = R^-1 g (back substitution) and x += V y, on the device
    LAUNCH(D, k_gmres_lsq, 1, 32, 0, m, D.gR, D.gg, D.gst, D.coef);
    LAUNCH(D, k_multiaxpy_dev, grid_for(N), 256, 0, N, D.gst, D.V, N, D.coef, 1.0, D.gx);
    R.its += st.j;
    R.relres = st.res / bn;
    if (st.done && st.res <= target) {
      R.converged = true;
      break;
    }
    // restart: r = b - A x
    tangent(c, D.gx, D.t1);
    LAUNCH(D, k_axpby, grid_for(N), 256, 0, N, 1.0, b, -1.0, D.t1, r);
    rn = norm2(D, N, r);
    R.relres = rn / bn;
    if (rn <= target) {
      R.converged = true;
      break;
    }
    if (st.done) break;
  }
  return R;
}

}  // namespace

int solve(Context& c, double* u_user, int u_dev, nls_report* rep) {
  Dev& D = *c.dev;
  nls_report rp;
  std::memset(&rp, 0, sizeof(rp));
  rp.first_failed_subdomain = -1;
  int status = NLS_OK;
  const int64_t N = c.N;
  const int64_t launches0 = D.launches;
  try {
    CK(cudaSetDevice(c.device));
    D.prof = c.opt.profile_kernels != 0;
    // a solve depends on its inputs only: the coarse factorization is reused across the outer
    // iterations of this call, never from an earlier one
    D.coarse_fact_valid = false;
    D.ainv_valid = false;
    D.local_factors_valid = false;
    D.local_reuse_active = c.opt.local_reuse != 0;
    struct ReuseScope {  // chord steps only inside this solve, never in a later nls_eval_Fx
      Dev& d;
      ~ReuseScope() { d.local_reuse_active = false; }
    } reuse_scope{D};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, D.s));
    auto w0 = std::chrono::steady_clock::now();
    CK(cudaMemcpyAsync(D.u, u_user, sizeof(double) * N, u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, D.s));
    LAUNCH(D, k_set_dirichlet, grid_for(N), 256, 0, N, D.free_dof, D.ubc, D.u);
    double t_inner = 0, t_coarse = 0, t_gmres = 0;
    const int L = std::max(1, c.opt.load_steps);
    double nF = INFINITY;
    // F_x at a point, with the statistics of its local and coarse solves
    auto eval_fx = [&](const double* x, double load) {
      FxInfo f = evaluate_Fx(c, x, load, &t_inner, &t_coarse);
      rp.subdomain_newton_steps += f.local_its;
      rp.local_chord_steps += f.local_chord;
      rp.coarse_newton_steps += f.coarse_its;
      rp.local_failures += f.local_failures;
      if (rp.first_failed_subdomain < 0) rp.first_failed_subdomain = f.first_failed;
      return f;
    };
    for (int step = 1; step <= L && status == NLS_OK; ++step) {
      const double load = (double)step / L;
      bool have_fx = false;  // D.Fx and the tangent data belong to D.u (from the backtracking)
      FxInfo fi;
      for (int k = 0;; ++k) {
        global_residual(c, D.u, D.F, load);
        nF = norm2(D, N, D.F);
        if (c.opt.verbose) std::fprintf(stderr, "[nls] load %.3f outer %d ||F|| = %.3e\n", load, k, nF);
        if (!std::isfinite(nF)) {
          status = NLS_E_DIVERGED;
          break;
        }
        if (nF < c.opt.outer_atol) break;
        if (k >= c.opt.outer_maxit) {
          status = NLS_W_NOT_CONVERGED;
          break;
        }
        if (!have_fx) {
          if (c.opt.coarse_rebuild && c.opt.coupling != NLS_COUPLING_ONE && c.coarse_kind == NLS_COARSE_RGDSW) {
            // the coarse basis from the current tangent: P_0 changes, so does every A_0
            coarse_extension(c, D.u);
            D.coarse_fact_valid = false;
            D.ainv_valid = false;
          }
          D.outer_k = k;
          fi = eval_fx(D.u, load);
          D.outer_k = -1;
        }
        have_fx = false;
        if (fi.pivot_failure) {
          status = NLS_E_PIVOT;
          break;
        }
        const double fxn = norm2(D, N, D.Fx);
        if (fxn == 0.0) {
          // Every correction vanished.  With all local and coarse solves converged, ||F|| is below
          // what their stopping tests resolve: the outer iteration has converged as far as it can.
          // With failed solves (their corrections are dropped) it cannot progress: not converged.
          if (fi.local_failures > 0 || fi.coarse_status != ST_OK) status = NLS_W_NOT_CONVERGED;
          break;
        }
        auto g0 = std::chrono::steady_clock::now();
        GmresResult gr = gmres(c, D.Fx);
        sync(D);
        t_gmres += std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
        rp.gmres_iterations += gr.its;
        rp.outer_iterations += 1;
        if (c.opt.verbose)
          std::fprintf(stderr, "[nls]   ||Fx|| = %.3e gmres %d (rel %.2e) local its %lld coarse its %d\n", fxn, gr.its,
                       gr.relres, (long long)fi.local_its, fi.coarse_its);
        if (!c.opt.outer_backtrack) {
          LAUNCH(D, k_axpby, grid_for(N), 256, 0, N, 1.0, D.u, -1.0, D.gx, D.u);
          continue;
        }
        // Backtracking on ||F_x||: the first of alpha = 1, 1/2, ... (at most min(ls_trials, 5))
        // with ||F(u')|| < outer_atol or ||F_x(u')|| <= (1 - armijo alpha) ||F_x(u)||, u' = u - alpha
        // du; the last trial is taken otherwise.  An accepted trial's F_x and tangent data serve
        // the next outer iteration, so a full step costs nothing extra.
        const int trials = std::max(1, std::min(c.opt.ls_trials, 5));
        double alpha = 1.0;
        for (int t = 0; t < trials; ++t) {
          LAUNCH(D, k_axpby, grid_for(N), 256, 0, N, 1.0, D.u, -alpha, D.gx, D.ut);
          global_residual(c, D.ut, D.F, load);
          const double nFt = norm2(D, N, D.F);
          if (nFt < c.opt.outer_atol) break;
          D.outer_k = k + 1;  // a trial point: the next outer iterate
          const FxInfo ft = eval_fx(D.ut, load);
          D.outer_k = -1;
          const double fxt = norm2(D, N, D.Fx);
          if ((std::isfinite(fxt) && fxt <= (1.0 - c.opt.armijo * alpha) * fxn) || t + 1 == trials ||
              ft.pivot_failure) {
            fi = ft;
            have_fx = true;
            break;
          }
          alpha *= 0.5;
        }
        if (c.opt.verbose && alpha < 1.0) std::fprintf(stderr, "[nls]   outer step alpha = %.4g\n", alpha);
        std::swap(D.u, D.ut);
      }
    }
    rp.final_residual = nF;
    CK(cudaMemcpyAsync(u_user, D.u, sizeof(double) * N, u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D.s));
    CK(cudaEventRecord(e1, D.s));
    CK(cudaEventSynchronize(e1));
    tlu_check_solves(c);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - w0).count();
    rp.time_total_s = ms * 1e-3;
    rp.time_inner_s = t_inner;
    rp.time_coarse_s = t_coarse;
    rp.time_gmres_s = t_gmres;
    rp.time_other_s = std::max(0.0, wall - t_inner - t_coarse - t_gmres);
    D.prof_flush();
  } catch (const DeviceTimeout& ex) {
    c.last_error = ex.what();
    status = NLS_E_DEVICE_TIMEOUT;
  } catch (const CudaFailure& ex) {
    c.last_error = ex.what();
    status = NLS_E_CUDA;
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    status = NLS_E_ARG;
  }
  rp.kernel_launches = D.launches - launches0;
  rp.status = status;
  if (rep) *rep = rp;
  return status;
}

int eval_F(Context& c, const double* u, double* F, int is_dev, double load) {
  Dev& D = *c.dev;
  try {
    CK(cudaMemcpyAsync(D.x, u, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, D.s));
    global_residual(c, D.x, D.F, load);
    CK(cudaMemcpyAsync(F, D.F, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D.s));
    sync(D);
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int eval_Fx(Context& c, const double* u, double* Fx, int is_dev, double load, int32_t* its, int32_t* st) {
  Dev& D = *c.dev;
  D.prof = c.opt.profile_kernels != 0;
  try {
    CK(cudaMemcpyAsync(D.u, u, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, D.s));
    FxInfo fi = evaluate_Fx(c, D.u, load, nullptr, nullptr);
    CK(cudaMemcpyAsync(Fx, D.Fx, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D.s));
    if (its) CK(cudaMemcpyAsync(its, D.ov.its, sizeof(int32_t) * c.ov.count, cudaMemcpyDeviceToHost, D.s));
    if (st) CK(cudaMemcpyAsync(st, D.ov.status, sizeof(int32_t) * c.ov.count, cudaMemcpyDeviceToHost, D.s));
    sync(D);
    if (fi.pivot_failure) return NLS_E_PIVOT;
  } catch (const DeviceTimeout& ex) {
    c.last_error = ex.what();
    return NLS_E_DEVICE_TIMEOUT;
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int apply_tangent(Context& c, const double* v, double* y, int is_dev) {
  Dev& D = *c.dev;
  if (!D.tangent_ready) {
    c.last_error = "nls_apply_tangent needs a preceding nls_eval_Fx";
    return NLS_E_ARG;
  }
  D.prof = c.opt.profile_kernels != 0;
  try {
    CK(cudaMemcpyAsync(D.t1, v, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, D.s));
    LAUNCH(D, k_mask, grid_for(c.N), 256, 0, c.N, D.free_dof, D.t1);
    CK(cudaMemcpyAsync(D.x, D.t1, sizeof(double) * c.N, cudaMemcpyDeviceToDevice, D.s));
    CK(cudaMemsetAsync(D.gx, 0, sizeof(double) * c.N, D.s));
    tangent(c, D.x, D.gx);
    CK(cudaMemcpyAsync(y, D.gx, sizeof(double) * c.N, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D.s));
    sync(D);
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int get_local_states(Context& c, double* w, int is_dev) {
  Dev& D = *c.dev;
  try {
    CK(cudaMemcpyAsync(w, D.ov.w, sizeof(double) * c.ov.total_n, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D.s));
    sync(D);
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int kernel_stats(const Context& c, int32_t cap, nls_kernel_stat* out, int32_t* n_out) {
  if (!c.dev) {
    *n_out = 0;
    return NLS_OK;
  }
  Dev& D = *c.dev;
  try {
    D.prof_flush();
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  int32_t n = 0;
  for (auto& st : D.stats) {
    if (out && n < cap) {
      out[n].name = st.name.c_str();
      out[n].launches = st.launches;
      out[n].total_ms = st.ms;
    }
    ++n;
  }
  // k_local_newton phases: CTA-milliseconds (sum over CTAs of thread 0's clock64 deltas)
  static const char* kPhaseNames[8] = {"phase:gather+residual", "phase:jacobian", "phase:band_lu",
                                       "phase:solve+refine",   "phase:line_search", "phase:tangent_jacobian",
                                       "phase:tangent_band_lu", "phase:output"};
  unsigned long long ph[8] = {0};
  try {
    CK(cudaMemcpy(ph, D.phase, sizeof(ph), cudaMemcpyDeviceToHost));
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  for (int k = 0; k < 8; ++k) {
    if (!ph[k]) continue;
    if (out && n < cap) {
      out[n].name = kPhaseNames[k];
      out[n].launches = 0;
      out[n].total_ms = (double)ph[k] / (double)D.clock_khz;
    }
    ++n;
  }
  *n_out = std::min(n, cap);
  return NLS_OK;
}

void reset_kernel_stats(Context& c) {
  if (!c.dev) return;
  try {
    c.dev->prof_flush();
    CK(cudaMemsetAsync(c.dev->phase, 0, sizeof(unsigned long long) * 8, c.dev->s));
  } catch (const std::exception&) {
  }
  c.dev->stats.clear();
}

int get_coarse_basis(const Context& c, double* P0) {
  if (c.coarse_kind != NLS_COARSE_RGDSW || !c.dev) return NLS_E_ARG;
  Dev& D = *c.dev;
  try {
    std::vector<double> vals(c.cs.p0_col.size());
    CK(cudaMemcpyAsync(vals.data(), D.p0_val, sizeof(double) * vals.size(), cudaMemcpyDeviceToHost, D.s));
    CK(cudaStreamSynchronize(D.s));
    std::memset(P0, 0, sizeof(double) * c.N * c.cs.N0);
    for (int64_t g = 0; g < c.N; ++g)
      for (int32_t k = c.cs.p0_rowptr[g]; k < c.cs.p0_rowptr[g + 1]; ++k) P0[(int64_t)c.cs.p0_col[k] * c.N + g] = vals[k];
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int guess_smooth(Context& c, const double* x, double load, const double* w, double* out) {
  if (!c.dev || !c.dev->guess) {
    c.last_error = "the learned-guess hooks need an attached network";
    return NLS_E_ARG;
  }
  Dev& D = *c.dev;
  try {
    const GuessProposal g = guess_smoothing(c);
    CK(cudaMemcpyAsync(D.x, x, sizeof(double) * c.N, cudaMemcpyHostToDevice, D.s));
    CK(cudaMemcpyAsync(D.ov.w, w, sizeof(double) * c.ov.total_n, cudaMemcpyHostToDevice, D.s));
    LocalArgs A = make_args(c, c.ov, D.ov);
    A.x = D.x;
    A.load = load;
    A.guess = D.ov.w;
    A.guess_diag = g.diag;
    A.guess_sweeps = g.sweeps;
    A.guess_omega = g.omega;
    A.out = D.ov.work;  // concatenated local vectors
    const size_t sm = sizeof(double) * ((size_t)c.ov.max_nt + c.ov.max_n) + 16;
    if (c.law == NLS_LAW_DIFFUSION) LAUNCH(D, k_guess_smooth<NLS_LAW_DIFFUSION>, c.ov.count, 128, sm, A);
    else LAUNCH(D, k_guess_smooth<NLS_LAW_NEOHOOKE>, c.ov.count, 128, sm, A);
    CK(cudaMemcpyAsync(out, D.ov.work, sizeof(double) * c.ov.total_n, cudaMemcpyDeviceToHost, D.s));
    sync(D);
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int get_coarse_matrix(const Context& c, double* A0) {
  if (c.coarse_kind != NLS_COARSE_RGDSW || !c.dev || !c.dev->A0) return NLS_E_ARG;
  Dev& D = *c.dev;
  try {
    CK(cudaMemcpyAsync(A0, D.A0, sizeof(double) * (size_t)c.cs.N0 * (2 * c.cs.b0 + 1), cudaMemcpyDeviceToHost, D.s));
    CK(cudaStreamSynchronize(D.s));
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

// The coarse factorization and solve on a given band matrix (parity hook and utility): a context
// with only the coarse problem, run on the legacy default stream and freed on return.
int band_solve(int device, int32_t n, int32_t b, const double* band, const double* rhs, double* x, int32_t precision,
               int32_t method, double* factors_out) {
  if (n < 1 || b < 0 || !band || !rhs || !x) return NLS_E_ARG;
  if ((precision != NLS_PREC_FP64 && precision != NLS_PREC_FP32_IR) || method < NLS_COARSE_FACTOR_AUTO ||
      method > NLS_COARSE_FACTOR_TILES)
    return NLS_E_ARG;
  Context c;
  c.device = device;
  c.stream = nullptr;
  nls_options_default(&c.opt);
  c.opt.coarse_precision = precision;
  c.opt.coarse_factor = method;
  c.coarse_kind = NLS_COARSE_RGDSW;
  c.cs.N0 = n;
  c.cs.b0 = b;
  int status = NLS_OK;
  try {
    if (b > kMaxSolveB0 || (!coarse_tiles(c) && b > kMaxBandB0)) return NLS_E_UNSUPPORTED;
    CK(cudaSetDevice(device));
    c.dev = new Dev();
    Dev& D = *c.dev;
    D.s = nullptr;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    D.nsm = prop.multiProcessorCount;
    D.smem_optin = prop.sharedMemPerBlockOptin;
    const bool f32 = fp32_coarse(c);
    const size_t fs = f32 ? sizeof(float) : sizeof(double);
    if (fs * (size_t)n > D.smem_optin || (!coarse_tiles(c) && coarse_factor_smem(c, f32) > D.smem_optin)) {
      device_free(c);
      return NLS_E_UNSUPPORTED;  // the one-CTA window or the solve vector exceeds shared memory
    }
    const size_t nw = (size_t)n * (2 * b + 1);
    D.A0 = D.alloc<double>(nw);
    CK(cudaMemcpyAsync(D.A0, band, sizeof(double) * nw, cudaMemcpyHostToDevice, D.s));
    const size_t ndinv = (size_t)packed_solve_entries(n, b);
    if (f32) {
      D.A0f = D.alloc<float>(nw);
      D.A0dinv = D.alloc<float>(ndinv);
    } else {
      D.A0f = D.alloc<double>(nw);
      D.A0dinv = D.alloc<double>(ndinv);
    }
    D.cstatus = D.alloc<int32_t>(1);
    D.cpart = D.alloc<double>(2 * (size_t)((n + 7) / 8));
    D.cflag = D.alloc<int>(2);
    CK(cudaMemsetAsync(D.cflag, 0, 2 * sizeof(int), D.s));
    D.cres = D.alloc<double>(n);
    D.g = D.alloc<double>(n);
    D.dc = D.alloc<double>(n);
    CK(cudaMemcpyAsync(D.g, rhs, sizeof(double) * n, cudaMemcpyHostToDevice, D.s));
    set_smem(k_coarse_factor<float>, D.smem_optin);
    set_smem(k_coarse_factor<double>, D.smem_optin);
    set_smem(k_coarse_band_solve<float>, D.smem_optin);
    set_smem(k_coarse_band_solve<double>, D.smem_optin);
    if (coarse_tiles(c)) tlu_prepare(c, f32);
    coarse_factor_launch(c);
    if (!coarse_status_ok(D)) {
      status = NLS_E_PIVOT;
    } else {
      coarse_solve(c, D.g, D.dc);
      CK(cudaMemcpyAsync(x, D.dc, sizeof(double) * n, cudaMemcpyDeviceToHost, D.s));
    }
    if (factors_out) {
      std::vector<float> f(f32 ? nw : 0);
      if (f32) CK(cudaMemcpyAsync(f.data(), D.A0f, sizeof(float) * nw, cudaMemcpyDeviceToHost, D.s));
      else CK(cudaMemcpyAsync(factors_out, D.A0f, sizeof(double) * nw, cudaMemcpyDeviceToHost, D.s));
      sync(D);
      if (f32)
        for (size_t k = 0; k < nw; ++k) factors_out[k] = (double)f[k];
    }
    sync(D);
    tlu_check_solves(c);
  } catch (const DeviceTimeout&) {
    status = NLS_E_DEVICE_TIMEOUT;
  } catch (const CudaFailure&) {
    status = NLS_E_CUDA;
  } catch (const std::bad_alloc&) {
    status = NLS_E_NOMEM;
  } catch (const std::exception&) {
    status = NLS_E_ARG;
  }
  device_free(c);
  return status;
}

// ------------------------------------------------------------------------------------------
// Local corrections without any allocation.
//
// Some callers cannot allocate device memory when they need the corrections: a solver step
// being recorded into a CUDA graph (cudaMalloc is not allowed while a stream is capturing),
// a host application whose memory manager owns every byte of the GPU, or a time-critical loop
// that must not risk the device-wide synchronisation cudaMalloc / cudaFree can cause.  For
// them the batched local-Newton kernel also runs on a fixed scratch area compiled into this
// library: a file-scope device array of kNoAllocScratchBytes that every GPU which loads the
// library keeps until the process exits.  Host code cannot use the array's name as a device
// address, so the address is looked up once per device with cudaGetSymbolAddress (on the
// first call on that device, which should therefore come before any stream capture) and then
// passed to the kernel.  All calls share the area and leave their contents in it; calls
// whose work overlaps on the GPU (different streams, or different contexts on one device)
// race on it.
// ------------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t noalloc_scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return cudaSuccess;
}

}  // namespace

int local_corrections_noalloc(Context& c, const double* x, double* Fx, int32_t* its_out, int32_t* status_out,
                              double load) {
  if (!c.is_setup || !c.dev) {
    c.last_error = "nls_local_corrections_noalloc needs a context after nls_setup";
    return NLS_E_ARG;
  }
  Dev& D = *c.dev;
  const LocalSet& s = c.ov;
  const bool f32 = fp32_local(c);
  // scratch plan: CSR values, band factors, packed solve operands, local states, work vectors,
  // its, status, work counter
  const size_t fbytes = f32 ? sizeof(float) : sizeof(double);
  size_t off = 0;
  const size_t o_csr = off;
  off = align_up(off + sizeof(double) * (size_t)s.total_nnz, 256);
  const size_t o_fac = off;
  off = align_up(off + fbytes * (size_t)s.total_factor, 256);
  const size_t o_dinv = off;
  off = align_up(off + fbytes * (size_t)s.total_dinv, 256);
  const size_t o_w = off;
  off = align_up(off + sizeof(double) * (size_t)s.total_n, 256);
  const size_t o_work = off;
  off = align_up(off + 3 * sizeof(double) * (size_t)s.total_n, 256);
  const size_t o_its = off;
  off = align_up(off + sizeof(int32_t) * (size_t)s.count, 256);
  const size_t o_st = off;
  off = align_up(off + sizeof(int32_t) * (size_t)s.count, 256);
  const size_t o_q = off;
  off = align_up(off + sizeof(int32_t), 256);
  if (off > kNoAllocScratchBytes) {
    c.last_error = "problem needs " + std::to_string(off) + " bytes of scratch; the allocation-free entry point has " +
                   std::to_string(kNoAllocScratchBytes);
    return NLS_E_ARG;
  }
  try {
    CK(cudaSetDevice(c.device));
    // per-launch event timing would create events: keep this path allocation free (the flag is
    // restored on return, so the context's profiling option is untouched)
    struct ProfScope {
      Dev& d;
      bool saved;
      ~ProfScope() { d.prof = saved; }
    } prof_scope{D, D.prof};
    D.prof = false;
    void* base = nullptr;
    CK(noalloc_scratch_address(c.device, &base));
    unsigned char* sc = (unsigned char*)base;
    LocalArgs A = make_args(c, s, D.ov);
    A.csr = (double*)(sc + o_csr);
    A.factor = sc + o_fac;
    A.dinv = sc + o_dinv;
    A.wbuf = (double*)(sc + o_w);
    A.work = (double*)(sc + o_work);
    A.work_stride = s.total_n;
    A.its = its_out ? its_out : (int32_t*)(sc + o_its);
    A.status = status_out ? status_out : (int32_t*)(sc + o_st);
    A.queue = (int32_t*)(sc + o_q);
    A.chord = nullptr;  // no chord steps here: the context's counters stay as they are
    A.reuse = 0;
    A.x = x;
    A.out = Fx;
    A.load = load;
    A.guess = nullptr;
    A.want_tangent = 0;
    // the work counter must start at zero; the rest of the area is written before it is read
    CK(cudaMemsetAsync(A.queue, 0, sizeof(int32_t), D.s));
    LAUNCH(D, k_mask, grid_for(c.N), 256, 0, c.N, D.free_dof, Fx);
    dispatch_local_newton(c, s, A, local_threads(c));
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

void options_changed(Context& c) {
  if (!c.dev) return;
  c.dev->coarse_fact_valid = false;
  c.dev->ainv_valid = false;
  c.dev->reset_graphs();
}

int get_tuning(const Context& c, nls_tuning* out) {
  std::memset(out, 0, sizeof(*out));
  out->newton_threads = local_threads(c);
  out->apply_threads = c.dev ? apply_threads(c) : std::max(64, min_local_threads(c));
  if (c.dev) {
    out->newton_tuned = c.dev->newton_tuned ? 1 : 0;
    out->apply_tuned = c.dev->apply_tuned ? 1 : 0;
    out->newton_ms[0] = c.dev->newton_ms[0];
    out->newton_ms[1] = c.dev->newton_ms[1];
    for (auto g : c.dev->it_exec) out->graphs_captured += g ? 1 : 0;
    out->coarse_threads = c.dev->coarse_T;
  }
  return NLS_OK;
}

}  // namespace nls
