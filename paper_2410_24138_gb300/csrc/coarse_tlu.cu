// Tiled band LU of the coarse matrix A_0 = P_0^T DF P_0 of Eq. 9, and the coarse solves with its
// factors (sm_103a).
//
// The coarse problem of the large workloads has tens of thousands of coarse dofs and a half
// bandwidth of several hundred (N_0 = 23,376, b_0 = 389 for the 2048^2 Neo-Hooke mesh), far
// beyond a factorization whose sliding window sits in one CTA's shared memory.  Here the band
// is cut into square tiles and factored without pivoting, right-looking, one tile column per
// step, across many CTAs:
//
//   step k:  A_kk = L_kk U_kk                      (every panel CTA, in registers, blocked by
//                                                   32-column groups)
//            L_ik = A_ik U_kk^-1,  U_kj = L_kk^-1 A_kj   (i, j = k+1 .. k+TB; row slabs per CTA)
//            A_ij -= L_ik U_kj                     (i, j = k+1 .. k+TB; one CTA per tile)
//
// FP32 factors (the chosen form) use 128 x 128 tiles and do the trailing products on the tensor
// cores: tcgen05.mma kind::tf32 from operands staged by TMA (cp.async.bulk.tensor) in the
// 128-byte swizzled layout, each FP32 operand split into TF32 high and low parts so that the
// three products hi*hi + hi*lo + lo*hi carry FP32 accuracy, accumulated in FP32 in TMEM.
// FP64 factors (the plain form) use 64 x 64 tiles and SIMT updates split into row slabs (the
// part has no FP64 tensor path).  Tiles to the right of the diagonal are stored transposed, so
// that both operands of every product are read along K:  for a tile on or below the diagonal
// Out[r][c] -= sum_t L_ik[r][t] (U_kj^T)[c][t], above it (Out^T)[c][r] -= sum_t (U_kj^T)[c][t]
// L_ik[r][t] -- in either case Out[a][b] -= sum_t P[a][t] Q[b][t] with P, Q stored rows.
//
// Solves (FP32 factors).  After the factorization the diagonal tiles are inverted (one CTA per
// tile) and the products M_tk = L_tt^-1 L_t,t-k and N_tk = U_tt^-1 U_t,t+k (k = 1 .. TB) are
// formed on the tensor cores, so that forward and backward substitution become, tile row by
// tile row,
//   y_t = L_tt^-1 g_t - sum_k M_tk y_{t-k},      x_t = U_tt^-1 y_t - sum_k N_tk x_{t+k}:
// one independent GEMV per row of the tile.  One cluster of 8 CTAs runs a solve: each CTA owns
// 16 rows of every tile, loads the next step's operand rows into registers while it finishes the
// current step, and sends its rows of y_t (x_t) into every CTA's shared memory (distributed shared
// memory, st.async completing on that step's mbarrier in the receiver), so that a step waits only
// for the tile it needs.  Every coarse solve is refined in FP64 against the band A_0 by the caller.
//
// The factors are also written in the band layout of the one-CTA factorization and packed into
// its triangular-solve operands (the explicit coarse inverse is built from those).
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <stdexcept>
#include <string>

#include "dev_state.cuh"
#include "device.cuh"
#include "nls_internal.h"
#include "tcgen05.cuh"

namespace nls {

namespace {

namespace cg = cooperative_groups;

__host__ __device__ inline int64_t tile_slot(int i, int j, int TB) { return (int64_t)i * (2 * TB + 1) + (j - i + TB); }

// Tile indices of the FP32 pool (one allocation, one tensor map): factor tiles, then the inverted
// diagonal tiles, the transposed L tiles, and the solve products M and N.
struct PoolIdx {
  int64_t inv, lt, m, n, total;
};
__host__ __device__ inline PoolIdx pool_index(int NT, int TB) {
  PoolIdx p;
  p.inv = (int64_t)NT * (2 * TB + 1);     // L_tt^-1 at inv + t, U_tt^-1 at inv + NT + t
  p.lt = p.inv + 2 * (int64_t)NT;         // (L_t,t-k)^T at lt + t TB + k - 1
  p.m = p.lt + (int64_t)NT * TB;          // M_tk at m + t TB + k - 1
  p.n = p.m + (int64_t)NT * TB;           // N_tk at n + t TB + k - 1
  p.total = p.n + (int64_t)NT * TB;
  return p;
}

// ---- A_0 (FP64 band, row-major, 2 b0 + 1 per row) -> tiles; rows and columns past N0 get the
// identity, so the padded matrix factors to the same leading factors ----------------------------
template <typename FT, int TS>
__global__ void k_tlu_init(int N0, int b0, int NT, int TB, const double* __restrict__ A0, FT* __restrict__ T) {
  const int SW = 2 * TB + 1, W = 2 * b0 + 1;
  const int64_t per = (int64_t)TS * TS, total = (int64_t)NT * SW * per;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / per;
    const int e = (int)(idx - s * per);
    const int i = (int)(s / SW), j = i + (int)(s % SW) - TB;
    int r = e / TS, c = e % TS;
    if (j > i) {  // stored transposed: position [p][q] holds entry (q, p)
      const int t = r;
      r = c;
      c = t;
    }
    FT v = (FT)0;
    if (j >= 0 && j < NT) {
      const int64_t R = (int64_t)i * TS + r, C = (int64_t)j * TS + c;
      if (R < N0 && C < N0) {
        const int64_t d = C - R + b0;
        if (d >= 0 && d < W) v = (FT)A0[R * W + d];
      } else if (R == C) {
        v = (FT)1;
      }
    }
    T[idx] = v;
  }
}

// ---- panel step ------------------------------------------------------------------------------
// Grid: 2 TB panels x NS row slabs (SLAB = TS / NS rows each).  Every CTA with work factors the
// diagonal tile (k, k) in shared memory (no pivoting; L scaled, U with its diagonal); CTA 0
// stores it in DG[k] and flags a zero or non-finite pivot.  Panel p < TB is the L tile
// (k+1+p, k): X := X U_kk^-1 on rows of the tile; panel p >= TB is the U tile (k, k+1+p-TB),
// stored transposed: X := X L_kk^-T on rows of the stored transpose.  Both are X := X M^-1 with
// M upper triangular.  The diagonal tile's LU and the slab's solve are both blocked by 32-column
// groups: one barrier per column inside a group, a rank-32 update of the rest after it.  With LT
// given, an L tile is also written transposed there (the B operand of M_tk for the solves).
template <typename FT>
__device__ inline FT rcp(FT x) {
  if constexpr (sizeof(FT) == 4) return __frcp_rn(x);
  else return (FT)1 / x;
}

template <typename FT, int TS, int NS>
__global__ void __launch_bounds__(512) k_tlu_panel(int k, int NT, int TB, FT* __restrict__ T, FT* __restrict__ DG,
                                                   FT* __restrict__ LT, int32_t* status) {
  // 512 threads as 16 x 32: thread (ty, tx) keeps the entries (ty + 16 a, tx + 32 b) of the tile
  // in registers (RA x CB of them); one elimination step only passes the pivot row and column
  // through shared memory (double-buffered by the step's parity: one barrier per step).
  constexpr int SLAB = TS / NS, LD = TS + 1, RA = TS / 16, CB = TS / 32, SA = SLAB / 16;
  static_assert(SLAB % 16 == 0 && TS % 32 == 0, "panel tiling");
  extern __shared__ __align__(16) unsigned char smem[];
  FT* Dg = (FT*)smem;           // TS x LD: the factored diagonal tile (for the slab solve)
  FT* rpiv = Dg + TS * LD;      // TS reciprocal pivots
  FT* rowbuf = rpiv + TS;       // 2 x TS
  FT* colbuf = rowbuf + 2 * TS; // 2 x TS
  __shared__ int s_bad;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int p = blockIdx.x / NS, q = blockIdx.x % NS;
  const bool lower = p < TB;
  const int other = k + 1 + (lower ? p : p - TB);  // the panel's tile row (L) or column (U)
  const bool has_panel = other < NT;
  if (!has_panel && blockIdx.x != 0) return;
  const FT* Akk = T + tile_slot(k, k, TB) * TS * TS;
  FT R[RA][CB];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < CB; ++b) R[a][b] = Akk[(ty + 16 * a) * TS + tx + 32 * b];
  if (tid == 0) s_bad = 0;
  // Blocked right-looking LU over the 32-column panels j of the tile.  Row r = ty + 16 a is the
  // same in a whole warp and column c = tx + 32 b is lane tx of column group b, so panel j is the
  // register column R[.][j] and its 32 pivot rows are a = 2j, 2j + 1.  For each pivot t of the
  // panel: rows below t update their panel column and, inside the panel's own 32 rows, also the
  // columns right of the panel (which makes those rows U12 = L11^-1 A12); then the rows below the
  // panel take the rank-32 product A22 -= L21 U12 at once, L21 from warp shuffles (row r's
  // multipliers sit in the lanes of its warp) and U12 through shared memory.
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    for (int t = 32 * j; t < 32 * j + 32; ++t) {
      FT* rb = rowbuf + (t & 1) * TS;
      FT* cb = colbuf + (t & 1) * TS;
#pragma unroll
      for (int a = 0; a < RA; ++a)
        if (ty + 16 * a == t) {
#pragma unroll
          for (int b = j; b < CB; ++b) rb[tx + 32 * b] = R[a][b];
        }
      if (tx == t - 32 * j) {
#pragma unroll
        for (int a = 0; a < RA; ++a) cb[ty + 16 * a] = R[a][j];
      }
      __syncthreads();
      const FT piv = rb[t];
      const FT rp = rcp<FT>(piv);
      if (tid == 0) {
        rpiv[t] = rp;
        if (!(piv != (FT)0) || !isfinite((double)piv)) s_bad = 1;
      }
#pragma unroll
      for (int a = 0; a < RA; ++a) {
        const int r = ty + 16 * a;
        if (r > t) {  // warp-uniform
          const FT l = cb[r] * rp;
          const int c = tx + 32 * j;
          if (c > t) R[a][j] -= l * rb[c];
          else if (c == t) R[a][j] = l;  // the multiplier of L
          if (a == 2 * j || a == 2 * j + 1) {  // the panel's own rows: U12
#pragma unroll
            for (int b = j + 1; b < CB; ++b) R[a][b] -= l * rb[tx + 32 * b];
          }
        }
      }
    }
    if (j + 1 < CB) {
      // U12 (rows 32 j .. 32 j + 31, columns right of the panel) into shared memory (Dg serves as
      // scratch until the end), then A22 -= L21 U12 on the rows below the panel
#pragma unroll
      for (int a = 2 * j; a < 2 * j + 2; ++a)
#pragma unroll
        for (int b = j + 1; b < CB; ++b) Dg[(ty + 16 * (a - 2 * j)) * LD + tx + 32 * b] = R[a][b];
      __syncthreads();
      for (int kk = 0; kk < 32; ++kk) {
        FT l[RA];
#pragma unroll
        for (int a = 2 * j + 2; a < RA; ++a) l[a] = __shfl_sync(0xffffffffu, R[a][j], kk);
#pragma unroll
        for (int b = j + 1; b < CB; ++b) {
          const FT u = Dg[kk * LD + tx + 32 * b];
#pragma unroll
          for (int a = 2 * j + 2; a < RA; ++a) R[a][b] -= l[a] * u;
        }
      }
      __syncthreads();  // U12 read by every warp before the next panel's rows overwrite the scratch
    }
  }
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < CB; ++b) Dg[(ty + 16 * a) * LD + tx + 32 * b] = R[a][b];
  __syncthreads();
  if (blockIdx.x == 0) {
    FT* out = DG + (int64_t)k * TS * TS;
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < CB; ++b) out[(ty + 16 * a) * TS + tx + 32 * b] = R[a][b];
    if (tid == 0 && s_bad) atomicExch(status, (int32_t)ST_PIVOT);
  }
  if (!has_panel) return;
  // X := X M^-1 on the slab's rows, M = U_kk (lower panel) or L_kk^T (upper panel, unit diagonal)
  FT* P = T + (lower ? tile_slot(other, k, TB) : tile_slot(k, other, TB)) * TS * TS + (int64_t)q * SLAB * TS;
  FT X[SA][CB];
  {
#pragma unroll
    for (int a = 0; a < SA; ++a)
#pragma unroll
      for (int b = 0; b < CB; ++b) X[a][b] = P[(ty + 16 * a) * TS + tx + 32 * b];
    // blocked over the 32-column groups j: column by column inside the group (one barrier per
    // column, only the group's register column X[.][j] changes), then the columns right of the
    // group take X[:, right] -= X[:, group] M[group, right] at once (the row's group values from
    // warp shuffles, M from the factored tile)
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      for (int t = 32 * j; t < 32 * j + 32; ++t) {
        FT* cb = colbuf + (t & 1) * TS;
        const FT rt = lower ? rpiv[t] : (FT)1;
        if (tx == t - 32 * j) {
#pragma unroll
          for (int a = 0; a < SA; ++a) cb[ty + 16 * a] = X[a][j] * rt;
        }
        const int c = tx + 32 * j;
        const FT m = (c > t) ? (lower ? Dg[t * LD + c] : Dg[c * LD + t]) : (FT)0;
        __syncthreads();
#pragma unroll
        for (int a = 0; a < SA; ++a) {
          const FT x = cb[ty + 16 * a];
          if (c > t) X[a][j] -= x * m;
          else if (c == t) X[a][j] = x;  // final value of column t
        }
      }
      if (j + 1 < CB) {
        for (int kk = 0; kk < 32; ++kk) {
          FT xv[SA];
#pragma unroll
          for (int a = 0; a < SA; ++a) xv[a] = __shfl_sync(0xffffffffu, X[a][j], kk);
          const int k = 32 * j + kk;
#pragma unroll
          for (int b = j + 1; b < CB; ++b) {
            const int c = tx + 32 * b;
            const FT m = lower ? Dg[k * LD + c] : Dg[c * LD + k];
#pragma unroll
            for (int a = 0; a < SA; ++a) X[a][b] -= xv[a] * m;
          }
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < SA; ++a)
#pragma unroll
    for (int b = 0; b < CB; ++b) P[(ty + 16 * a) * TS + tx + 32 * b] = X[a][b];
  if (lower && LT) {  // (L_other,k)^T: entry [c][r] = L[r][c]
    FT* out = LT + ((int64_t)other * TB + (other - k - 1)) * TS * TS;
#pragma unroll
    for (int a = 0; a < SA; ++a)
#pragma unroll
      for (int b = 0; b < CB; ++b) out[(int64_t)(tx + 32 * b) * TS + q * SLAB + ty + 16 * a] = X[a][b];
  }
}

// ---- trailing update, SIMT (FP64 factors) ------------------------------------------------------
// Grid: TB x TB tiles x NS row slabs; Out[a][b] -= sum_t P[a][t] Q[b][t] on rows a of the slab.
template <typename FT, int TS, int NS>
__global__ void __launch_bounds__(256) k_tlu_update_simt(int k, int NT, int TB, FT* __restrict__ T) {
  constexpr int SLAB = TS / NS, LD = TS + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  FT* Qs = (FT*)smem;     // TS x LD
  FT* Ps = Qs + TS * LD;  // SLAB x LD
  const int tile = blockIdx.x / NS, q = blockIdx.x % NS;
  const int i = k + 1 + tile / TB, j = k + 1 + tile % TB;
  if (i >= NT || j >= NT) return;
  const int64_t sP = (i >= j) ? tile_slot(i, k, TB) : tile_slot(k, j, TB);
  const int64_t sQ = (i >= j) ? tile_slot(k, j, TB) : tile_slot(i, k, TB);
  const FT* P = T + sP * TS * TS + (int64_t)q * SLAB * TS;
  const FT* Q = T + sQ * TS * TS;
  FT* O = T + tile_slot(i, j, TB) * TS * TS + (int64_t)q * SLAB * TS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < TS * TS; e += nt) Qs[(e / TS) * LD + e % TS] = Q[e];
  for (int e = tid; e < SLAB * TS; e += nt) Ps[(e / TS) * LD + e % TS] = P[e];
  __syncthreads();
  for (int e = tid; e < SLAB * TS; e += nt) {
    const int a = e / TS, b = e % TS;
    FT acc = 0;
#pragma unroll 8
    for (int t = 0; t < TS; ++t) acc += Ps[a * LD + t] * Qs[b * LD + t];
    O[e] -= acc;
  }
}

// ---- 128 x 128 x 128 tile products on the tensor cores --------------------------------------------
// D = A B^T for the operand tiles at tensor-map rows yA and yB (row-major, K = 128 contiguous), in
// four chunks of 32 values staged by TMA (SW128, 16 KB each) into a two-stage ring; the threads
// split every value into TF32 hi + lo in place; one thread issues the 3 x 4 MMAs of a chunk
// (K = 8 each) into a 128 x 128 FP32 accumulator in TMEM; the epilogue (warp w: rows 32 w ..
// 32 w + 31) subtracts D from `out` (subtract) or stores it there.  Four warps per CTA.
constexpr int kTcTS = 128;
constexpr int kTcChunkBytes = 128 * 32 * 4;      // one operand chunk: 128 rows x 32 FP32
constexpr int kTcStageBytes = 4 * kTcChunkBytes;  // A hi, B hi, A lo, B lo
constexpr size_t kTcSmem = 2 * kTcStageBytes + 1024;

__device__ void tile_product(const CUtensorMap* map, int yA, int yB, float* __restrict__ out, bool subtract,
                             int32_t* status) {
  using namespace tc;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_tma[2], bar_mma[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_tma[0], 1);
    mbar_init(&bar_tma[1], 1);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    mbar_init_fence();
    s_fail = 0;
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, 128);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  auto buf = [&](int st, int which) { return (float*)(sm + st * kTcStageBytes + which * kTcChunkBytes); };
  auto issue = [&](int kc) {
    const int st = kc & 1;
    mbar_arrive_expect_tx(&bar_tma[st], 2 * kTcChunkBytes);
    tma_load_2d(buf(st, 0), map, 32 * kc, yA, &bar_tma[st]);
    tma_load_2d(buf(st, 1), map, 32 * kc, yB, &bar_tma[st]);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  constexpr uint32_t idesc = idesc_tf32(128, 128);
  for (int kc = 0; kc < 4; ++kc) {
    const int st = kc & 1;
    const uint32_t par = (uint32_t)(kc >> 1) & 1u;
    if (!mbar_wait(&bar_tma[st], par)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    {
      float4* ah = (float4*)buf(st, 0);
      float4* bh = (float4*)buf(st, 1);
      float4* al = (float4*)buf(st, 2);
      float4* bl = (float4*)buf(st, 3);
      for (int e = tid; e < kTcChunkBytes / 16; e += 128) {
        float4 x = ah[e], h, l;
        split_tf32(x.x, h.x, l.x);
        split_tf32(x.y, h.y, l.y);
        split_tf32(x.z, h.z, l.z);
        split_tf32(x.w, h.w, l.w);
        ah[e] = h;
        al[e] = l;
        x = bh[e];
        split_tf32(x.x, h.x, l.x);
        split_tf32(x.y, h.y, l.y);
        split_tf32(x.z, h.z, l.z);
        split_tf32(x.w, h.w, l.w);
        bh[e] = h;
        bl[e] = l;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint64_t ah = desc_sw128(buf(st, 0)), bh = desc_sw128(buf(st, 1));
      const uint64_t al = desc_sw128(buf(st, 2)), bl = desc_sw128(buf(st, 3));
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint64_t off = (uint64_t)(32 * s) >> 4;  // K = 8 FP32 = 32 bytes into the swizzled row
        mma_tf32(tmem, al + off, bh + off, idesc, (kc | s) ? 1u : 0u);
        mma_tf32(tmem, ah + off, bl + off, idesc, 1u);
        mma_tf32(tmem, ah + off, bh + off, idesc, 1u);
      }
      mma_commit(&bar_mma[st]);
      if (kc + 2 < 4) {
        // the stage is reused for chunk kc + 2 once the MMAs reading it have completed
        if (mbar_wait(&bar_mma[st], par)) issue(kc + 2);
        else s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) break;
  }
  // the last commit (chunk 3: stage 1, its second phase) completes after every MMA
  if (!s_fail && !mbar_wait(&bar_mma[1], 1u)) s_fail = 1;
  __syncthreads();
  fence_after_sync();
  if (!s_fail) {
    float4* orow = (float4*)(out + (int64_t)(32 * warp + lane) * kTcTS);
#pragma unroll 1
    for (int c0 = 0; c0 < kTcTS; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        float4 o;
        if (subtract) {
          o = orow[c0 / 4 + q4];
          o.x -= v[4 * q4];
          o.y -= v[4 * q4 + 1];
          o.z -= v[4 * q4 + 2];
          o.w -= v[4 * q4 + 3];
        } else {
          o = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
        }
        orow[c0 / 4 + q4] = o;
      }
    }
  } else if (tid == 0) {
    atomicExch(status, (int32_t)ST_TIMEOUT);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// Trailing update of factorization step k: one CTA per tile (i, j), i, j = k+1 .. k+TB.
__global__ void __launch_bounds__(128, 1) k_tlu_update_tc(const __grid_constant__ CUtensorMap map, int k, int NT,
                                                           int TB, float* __restrict__ T, int32_t* status) {
  const int i = k + 1 + (int)blockIdx.x / TB, j = k + 1 + (int)blockIdx.x % TB;
  if (i >= NT || j >= NT) return;
  const int64_t sP = (i >= j) ? tile_slot(i, k, TB) : tile_slot(k, j, TB);
  const int64_t sQ = (i >= j) ? tile_slot(k, j, TB) : tile_slot(i, k, TB);
  tile_product(&map, (int)(sP * kTcTS), (int)(sQ * kTcTS), T + tile_slot(i, j, TB) * kTcTS * kTcTS, true, status);
}

// The solve products: CTA (which, t, k): M_tk = L_tt^-1 L_t,t-k (B operand: (L_t,t-k)^T, whose
// rows are K) or N_tk = U_tt^-1 U_t,t+k (B operand: the stored transpose of U_t,t+k).
__global__ void __launch_bounds__(128, 1) k_tile_solve_products(const __grid_constant__ CUtensorMap map, int NT,
                                                                 int TB, float* __restrict__ pool, int32_t* status) {
  const PoolIdx P = pool_index(NT, TB);
  const int per = NT * TB;
  const bool is_n = (int)blockIdx.x >= per;
  const int r = (int)blockIdx.x - (is_n ? per : 0);
  const int t = r / TB, k = r % TB + 1;
  if (!is_n && t - k < 0) return;
  if (is_n && t + k >= NT) return;
  const int64_t a = is_n ? P.inv + NT + t : P.inv + t;
  const int64_t b = is_n ? tile_slot(t, t + k, TB) : P.lt + (int64_t)t * TB + k - 1;
  const int64_t o = (is_n ? P.n : P.m) + (int64_t)t * TB + k - 1;
  tile_product(&map, (int)(a * kTcTS), (int)(b * kTcTS), pool + o * kTcTS * kTcTS, false, status);
}

// ---- inverses of the factored diagonal tiles (FP32, 128 x 128) ------------------------------------
// One CTA of 1024 threads per tile: threads 0..511 form L_tt^-1 (unit lower), 512..1023 U_tt^-1.
// Four lanes own one column of the inverse and run its substitution over all rows (forward for
// L, backward for U), each lane a quarter of every dot product, reduced by shuffles: no barrier
// between rows, since a column depends on its own earlier entries only.
__global__ void __launch_bounds__(1024) k_tile_inverses(int NT, const float* __restrict__ DG, float* __restrict__ INVL,
                                                        float* __restrict__ INVU) {
  constexpr int TS = 128, LD = TS + 1;
  extern __shared__ __align__(16) float smf[];
  float* Dg = smf;
  float* XL = Dg + TS * LD;
  float* XU = XL + TS * LD;
  const int t = blockIdx.x;
  const float* D = DG + (int64_t)t * TS * TS;
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) Dg[(e / TS) * LD + e % TS] = D[e];
  __syncthreads();
  const bool upper = threadIdx.x >= 512;
  const int tl = threadIdx.x & 511, c = tl >> 2, part = tl & 3;
  float* X = upper ? XU : XL;
  if (!upper) {
    for (int i = 0; i < TS; ++i) {
      float s = 0.f;
      for (int k = part; k < i; k += 4) s += Dg[i * LD + k] * X[k * LD + c];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (part == 0) X[i * LD + c] = (i == c ? 1.f : 0.f) - s;
      __syncwarp();
    }
  } else {
    for (int i = TS - 1; i >= 0; --i) {
      float s = 0.f;
      for (int k = i + 1 + part; k < TS; k += 4) s += Dg[i * LD + k] * X[k * LD + c];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (part == 0) X[i * LD + c] = ((i == c ? 1.f : 0.f) - s) / Dg[i * LD + i];
      __syncwarp();
    }
  }
  __syncthreads();
  float* OL = INVL + (int64_t)t * TS * TS;
  float* OU = INVU + (int64_t)t * TS * TS;
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    OL[e] = XL[(e / TS) * LD + e % TS];
    OU[e] = XU[(e / TS) * LD + e % TS];
  }
}

// ---- the cluster solve -------------------------------------------------------------------------
// z = (accumulate ? z : 0) + A_0^-1 rhs with the tile products above, by one cluster of kSolveCL
// CTAs (see the head of this file).  Shared memory per CTA: the whole forward result y (every CTA
// keeps all of it: NT x 128 FP32), a ring of TB + 1 tiles of x, the current tile of rhs
// (double-buffered) and one mbarrier per step of each sweep.  CTA r solves rows 16 r .. 16 r + 15
// of every tile (two per warp) and sends them to every CTA of the cluster with st.async, which
// completes 8 bytes per warp on the receiver's mbarrier of that step (8 CTAs x 8 warps x 8 bytes =
// 512 bytes per step); a step waits only for the mbarrier of the tile it needs, not for a
// cluster-wide barrier.  Each mbarrier is used once (phase 0).  Ring slots of x are safe to
// overwrite: a CTA sends x_t only after x_{t+1} has arrived from every CTA, i.e. after every warp
// of the cluster has read what it needed from slot t mod (TB + 1).  Waits are bounded: a CTA that
// gives up sets *status = ST_TIMEOUT and stops waiting (its results are then garbage; the host
// raises).  With *skip set the kernel returns at once in every CTA (the flag is written by an
// earlier kernel, so all CTAs read the same value); `reset`, if given, is cleared.
constexpr int kSolveCL = 8;
constexpr int kSolveRows = kTcTS / kSolveCL;  // rows of every tile per CTA (two per warp)
constexpr int kSolveMaxTB = 4;                // TB of half bandwidths up to 480 (the solves' limit)

__device__ inline float dot4(const float4 a, const float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

__global__ void __cluster_dims__(kSolveCL, 1, 1) __launch_bounds__(256, 1)
    k_tile_solve(int N0, int NT, int TB, const float* __restrict__ pool, const double* __restrict__ rhs,
                 double* __restrict__ z, int accumulate, const int* skip, int* reset, int32_t* status) {
  if (skip && *skip) return;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) float sms[];
  float* y = sms;                                 // NT x 128
  float* xr = y + (int64_t)NT * kTcTS;            // (TB + 1) x 128 ring
  float* gt = xr + (kSolveMaxTB + 1) * kTcTS;     // 2 x 128 (double-buffered right-hand side)
  uint64_t* fb = (uint64_t*)(gt + 2 * kTcTS);     // NT forward-step barriers
  uint64_t* bb = fb + NT;                         // NT backward-step barriers
  const PoolIdx P = pool_index(NT, TB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = rank * kSolveRows + 2 * warp;  // this warp's rows within every tile
  if (reset && rank == 0 && threadIdx.x == 0) *reset = 0;
  constexpr int64_t TT = (int64_t)kTcTS * kTcTS;
  constexpr uint32_t kStepBytes = kSolveCL * kSolveRows * sizeof(float);
  if (threadIdx.x == 0) {
    for (int t = 0; t < 2 * NT; ++t) tc::mbar_init(fb + t, 1);
    tc::mbar_init_fence();
    for (int t = 0; t < 2 * NT; ++t) tc::mbar_arrive_expect_tx(fb + t, kStepBytes);
  }
  bool live = true;  // false once a wait gave up: no further waits
  auto wait = [&](uint64_t* bar) {
    if (live && !tc::mbar_wait_cluster(bar, 0)) {
      live = false;
      if (lane == 0) atomicExch(status, (int32_t)ST_TIMEOUT);
    }
  };
  // operand rows of one step into registers: [0] the diagonal inverse, [k] the k-th product
  float4 cur[kSolveMaxTB + 1][2], nxt[kSolveMaxTB + 1][2];
  auto load = [&](int t, bool fwd, float4 (&R)[kSolveMaxTB + 1][2]) {
    const float* D = pool + (fwd ? P.inv + t : P.inv + NT + t) * TT;
    R[0][0] = __ldg((const float4*)(D + (int64_t)row0 * kTcTS) + lane);
    R[0][1] = __ldg((const float4*)(D + (int64_t)(row0 + 1) * kTcTS) + lane);
#pragma unroll
    for (int k = 1; k <= kSolveMaxTB; ++k) {
      const bool ok = k <= TB && (fwd ? t - k >= 0 : t + k < NT);
      if (ok) {
        const float* M = pool + ((fwd ? P.m : P.n) + (int64_t)t * TB + k - 1) * TT;
        R[k][0] = __ldg((const float4*)(M + (int64_t)row0 * kTcTS) + lane);
        R[k][1] = __ldg((const float4*)(M + (int64_t)(row0 + 1) * kTcTS) + lane);
      } else {
        R[k][0] = R[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  // operand rows of the step kSolveL2 ahead into L2 (each lane one 128-byte line of its warp's
  // rows: 2 rows x (TB + 1) tiles x 4 lines), so that the register loads one step ahead hit L2
  auto l2_ahead = [&](int t, bool fwd) {
    const int tile = lane >> 3, rr = (lane >> 2) & 1, line = lane & 3;  // 4 tiles x 2 rows x 4 lines
    for (int k = tile; k <= TB; k += 4) {
      if (k > 0 && (fwd ? t - k < 0 : t + k >= NT)) continue;
      const float* base = pool + (k == 0 ? (fwd ? P.inv + t : P.inv + NT + t)
                                         : (fwd ? P.m : P.n) + (int64_t)t * TB + k - 1) * TT;
      const float* a = base + (int64_t)(row0 + rr) * kTcTS + 32 * line;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a)));
    }
  };
  // this warp's two solved rows of step t into CTA `lane`'s copy of `buf`, completing on its `bar`
  auto send = [&](float* buf, uint64_t* bar, float a0, float a1) {
    if (lane < kSolveCL) tc::st_async_f2(tc::cluster_addr(buf + row0, lane), a0, a1, tc::cluster_addr(bar, lane));
  };
  constexpr int kSolveL2 = 4;
  cl.sync();  // every CTA's barriers are initialised and armed before the first remote store
  // forward: y_t = L_tt^-1 g_t - sum_k M_tk y_{t-k}; the right-hand side of the next step is read
  // into a register during the current one (double-buffered tile gt)
  load(0, true, cur);
  for (int q = 1; q < kSolveL2 && q < NT; ++q) l2_ahead(q, true);
  float gnext = 0.f;
  if (threadIdx.x < kTcTS) gt[threadIdx.x] = threadIdx.x < N0 ? (float)rhs[threadIdx.x] : 0.f;
  __syncthreads();
  for (int t = 0; t < NT; ++t) {
    if (t + 1 < NT) load(t + 1, true, nxt);
    if (t + kSolveL2 < NT) l2_ahead(t + kSolveL2, true);
    if (threadIdx.x < kTcTS && t + 1 < NT) {
      const int64_t R = (int64_t)(t + 1) * kTcTS + threadIdx.x;
      gnext = R < N0 ? (float)rhs[R] : 0.f;
    }
    const float4 g4 = ((const float4*)(gt + (t & 1) * kTcTS))[lane];
    float a0 = dot4(cur[0][0], g4), a1 = dot4(cur[0][1], g4);
    // the terms of tiles that arrived in earlier steps first, then wait for y_{t-1}
#pragma unroll
    for (int k = 2; k <= kSolveMaxTB; ++k)
      if (k <= TB && t - k >= 0) {
        const float4 yv = ((const float4*)(y + (int64_t)(t - k) * kTcTS))[lane];
        a0 -= dot4(cur[k][0], yv);
        a1 -= dot4(cur[k][1], yv);
      }
    if (t >= 1) {
      wait(fb + t - 1);
      const float4 yv = ((const float4*)(y + (int64_t)(t - 1) * kTcTS))[lane];
      a0 -= dot4(cur[1][0], yv);
      a1 -= dot4(cur[1][1], yv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    send(y + (int64_t)t * kTcTS, fb + t, a0, a1);
    if (threadIdx.x < kTcTS && t + 1 < NT) gt[((t + 1) & 1) * kTcTS + threadIdx.x] = gnext;
    __syncthreads();  // the next step's right-hand side tile
#pragma unroll
    for (int k = 0; k <= kSolveMaxTB; ++k) cur[k][0] = nxt[k][0], cur[k][1] = nxt[k][1];
  }
  wait(fb + NT - 1);
  // backward: x_t = U_tt^-1 y_t - sum_k N_tk x_{t+k}
  const int RB = TB + 1;
  load(NT - 1, false, cur);
  for (int q = 1; q < kSolveL2 && NT - 1 - q >= 0; ++q) l2_ahead(NT - 1 - q, false);
  for (int t = NT - 1; t >= 0; --t) {
    if (t > 0) load(t - 1, false, nxt);
    if (t - kSolveL2 >= 0) l2_ahead(t - kSolveL2, false);
    const float4 yv = ((const float4*)(y + (int64_t)t * kTcTS))[lane];
    float a0 = dot4(cur[0][0], yv), a1 = dot4(cur[0][1], yv);
#pragma unroll
    for (int k = 2; k <= kSolveMaxTB; ++k)
      if (k <= TB && t + k < NT) {
        const float4 xv = ((const float4*)(xr + ((t + k) % RB) * kTcTS))[lane];
        a0 -= dot4(cur[k][0], xv);
        a1 -= dot4(cur[k][1], xv);
      }
    if (t + 1 < NT) {
      wait(bb + t + 1);  // x_{t+1} complete
      const float4 xv = ((const float4*)(xr + ((t + 1) % RB) * kTcTS))[lane];
      a0 -= dot4(cur[1][0], xv);
      a1 -= dot4(cur[1][1], xv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    send(xr + (t % RB) * kTcTS, bb + t, a0, a1);
    if (lane == 0) {
      const int64_t R0 = (int64_t)t * kTcTS + row0;
      if (R0 < N0) z[R0] = (accumulate ? z[R0] : 0.0) + (double)a0;
      if (R0 + 1 < N0) z[R0 + 1] = (accumulate ? z[R0 + 1] : 0.0) + (double)a1;
    }
#pragma unroll
    for (int k = 0; k <= kSolveMaxTB; ++k) cur[k][0] = nxt[k][0], cur[k][1] = nxt[k][1];
  }
  wait(bb);  // every remote store into this CTA has landed before it leaves
  cl.sync();
}

size_t tile_solve_smem(int NT) {
  return sizeof(float) * ((size_t)NT * kTcTS + (kSolveMaxTB + 3) * kTcTS) + 2 * sizeof(uint64_t) * (size_t)NT;
}

// ---- tiles -> band layout of the one-CTA factorization: d < b0 L (scaled), d = b0 the reciprocal
// pivot, d > b0 U -------------------------------------------------------------------------------
template <typename FT, int TS>
__global__ void k_tlu_to_band(int N0, int b0, int TB, const FT* __restrict__ T, const FT* __restrict__ DG,
                              FT* __restrict__ F) {
  const int W = 2 * b0 + 1;
  const int64_t total = (int64_t)N0 * W;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int R = (int)(idx / W), d = (int)(idx - (int64_t)R * W);
    const int C = R - b0 + d;
    FT v = (FT)0;
    if (C >= 0 && C < N0) {
      const int i = R / TS, j = C / TS, r = R % TS, c = C % TS;
      if (i == j) {
        const FT x = DG[(int64_t)i * TS * TS + r * TS + c];
        v = (r == c) ? (FT)1 / x : x;
      } else if (j < i) {
        v = T[tile_slot(i, j, TB) * TS * TS + r * TS + c];
      } else {
        v = T[tile_slot(i, j, TB) * TS * TS + c * TS + r];
      }
    }
    F[idx] = v;
  }
}

// packed triangular-solve operands from the band factors, 8 warps per CTA, blocks spread over CTAs
template <typename FT>
__global__ void __launch_bounds__(256) k_band_pack(int n, int b, const FT* __restrict__ F, FT* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smem[];
  dev::band_pack_solve_range<FT>(n, b, F, P, (FT*)smem, 8, blockIdx.x * 8, gridDim.x * 8);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

inline int grid_for_n(int64_t n, int threads = 256) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1216));
}

template <typename FT, int TS, int NS>
size_t panel_smem() {
  return sizeof(FT) * ((size_t)TS * (TS + 1) + 5 * (size_t)TS);
}
template <typename FT, int TS, int NS>
size_t update_simt_smem() {
  return sizeof(FT) * ((size_t)TS * (TS + 1) + (size_t)(TS / NS) * (TS + 1));
}
constexpr size_t kInvSmem = sizeof(float) * 3 * 128 * 129;

constexpr int kNS32 = 4, kNS64 = 4;  // row slabs per panel / update tile
constexpr int kTS64 = 64;

template <typename FT, int TS, int NS>
void tlu_factor_t(Context& c, TileLU& L) {
  Dev& D = *c.dev;
  const int N0 = c.cs.N0, b0 = c.cs.b0, NT = L.NT, TB = L.TB;
  const int64_t l0 = D.launches;
  FT* T = (FT*)L.T;
  FT* DG = (FT*)L.DG;
  const bool f32 = sizeof(FT) == 4;
  const PoolIdx P = pool_index(NT, TB);
  float* pool = (float*)L.T;
  CK(cudaMemsetAsync(D.cstatus, 0, sizeof(int32_t), D.s));
  const int64_t total = (int64_t)NT * L.SW * TS * TS;
  LAUNCH_NAMED(D, "k_tlu_init", (k_tlu_init<FT, TS>), grid_for_n(total), 256, 0, N0, b0, NT, TB, c.dev->A0, T);
  const size_t psm = panel_smem<FT, TS, NS>();
  FT* LT = f32 && L.solve_tiles ? (FT*)(pool + P.lt * TS * TS) : nullptr;
  for (int k = 0; k < NT; ++k) {
    LAUNCH_NAMED(D, "k_tlu_panel", (k_tlu_panel<FT, TS, NS>), 2 * TB * NS, 512, psm, k, NT, TB, T, DG, LT, D.cstatus);
    if (k + 1 < NT) {
      if constexpr (sizeof(FT) == 4) {
        LAUNCH_NAMED(D, "k_tlu_update_tc", k_tlu_update_tc, TB * TB, 128, kTcSmem, L.map, k, NT, TB, T, D.cstatus);
      } else {
        LAUNCH_NAMED(D, "k_tlu_update_simt", (k_tlu_update_simt<FT, TS, NS>), TB * TB * NS, 256,
                     (update_simt_smem<FT, TS, NS>()), k, NT, TB, T);
      }
    }
  }
  if constexpr (sizeof(FT) == 4) {
    if (L.solve_tiles) {
      LAUNCH_NAMED(D, "k_tile_inverses", k_tile_inverses, NT, 1024, kInvSmem, NT, (const float*)DG,
                   pool + P.inv * TS * TS, pool + (P.inv + NT) * TS * TS);
      LAUNCH_NAMED(D, "k_tile_solve_products", k_tile_solve_products, 2 * NT * TB, 128, kTcSmem, L.map, NT, TB, pool,
                   D.cstatus);
    }
  }
  const int64_t nb = (int64_t)N0 * (2 * b0 + 1);
  LAUNCH_NAMED(D, "k_tlu_to_band", (k_tlu_to_band<FT, TS>), grid_for_n(nb), 256, 0, N0, b0, TB, T, DG, (FT*)D.A0f);
  constexpr int BS = dev::SolveBlock<FT>::BS;
  const int nblk = (N0 + BS - 1) / BS;
  LAUNCH_NAMED(D, "k_band_pack", k_band_pack<FT>, (nblk + 7) / 8, 256, sizeof(FT) * 8 * BS * (BS + 1), N0, b0,
               (const FT*)D.A0f, (FT*)D.A0dinv);
  L.launches_per_factor = D.launches - l0;
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

// Storage, tensor map and kernel attributes of the tiled factorization of A_0 (at setup).
void tlu_prepare(Context& c, bool f32) {
  Dev& D = *c.dev;
  if (D.tlu) return;
  TileLU* L = new TileLU();
  D.tlu = L;
  L->f32 = f32;
  L->TS = f32 ? kTcTS : kTS64;
  L->NT = (c.cs.N0 + L->TS - 1) / L->TS;
  L->TB = std::max(1, (c.cs.b0 + L->TS - 1) / L->TS);
  L->SW = 2 * L->TB + 1;
  const size_t per = (size_t)L->TS * L->TS;
  if (f32) {
    L->solve_tiles = L->TB <= kSolveMaxTB && tile_solve_smem(L->NT) <= D.smem_optin;
    const PoolIdx P = pool_index(L->NT, L->TB);
    const int64_t tiles = L->solve_tiles ? P.total : (int64_t)L->NT * L->SW;
    L->T = D.alloc<float>((size_t)tiles * per);
    L->DG = D.alloc<float>((size_t)L->NT * per);
    L->solve_status = D.alloc<int32_t>(1);
    CK(cudaMemsetAsync(L->solve_status, 0, sizeof(int32_t), D.s));
    auto enc = tensor_map_encoder();
    if (!enc) throw std::runtime_error("cuTensorMapEncodeTiled is not available from the driver");
    const uint64_t rows = (uint64_t)tiles * L->TS;
    if (rows >= (1ull << 31)) throw std::runtime_error("coarse tile storage too large for one tensor map");
    cuuint64_t dims[2] = {(cuuint64_t)L->TS, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(L->TS * sizeof(float))};
    cuuint32_t box[2] = {32, (cuuint32_t)L->TS};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&L->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, L->T, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    allow_smem(k_tlu_panel<float, kTcTS, kNS32>, panel_smem<float, kTcTS, kNS32>());
    allow_smem(k_tlu_update_tc, kTcSmem);
    allow_smem(k_tile_solve_products, kTcSmem);
    allow_smem(k_tile_inverses, kInvSmem);
    if (L->solve_tiles) allow_smem(k_tile_solve, tile_solve_smem(L->NT));
    allow_smem(k_band_pack<float>, sizeof(float) * 8 * 32 * 33);
  } else {
    L->T = D.alloc<double>((size_t)L->NT * L->SW * per);
    L->DG = D.alloc<double>((size_t)L->NT * per);
    allow_smem(k_tlu_panel<double, kTS64, kNS64>, panel_smem<double, kTS64, kNS64>());
    allow_smem(k_tlu_update_simt<double, kTS64, kNS64>, update_simt_smem<double, kTS64, kNS64>());
    allow_smem(k_band_pack<double>, sizeof(double) * 8 * 16 * 17);
  }
}

void tlu_free(Context& c) {
  if (c.dev && c.dev->tlu) {
    delete c.dev->tlu;  // the device arrays are in Dev::allocs
    c.dev->tlu = nullptr;
  }
}

// Factor D.A0 (FP64 band) into D.A0f (band layout) and D.A0dinv (packed solve operands) -- and,
// for FP32 factors, the inverted diagonal tiles and solve products of the cluster solve; the
// status word D.cstatus receives ST_PIVOT for a zero or non-finite pivot, ST_TIMEOUT if a
// tensor-core tile gave up waiting for its operands.
void tlu_factor(Context& c) {
  TileLU& L = *c.dev->tlu;
  if (L.f32) tlu_factor_t<float, kTcTS, kNS32>(c, L);
  else tlu_factor_t<double, kTS64, kNS64>(c, L);
}

// z = (accumulate ? z : 0) + A_0^-1 rhs with the tile products (one cluster); false when the
// factorization has no solve tiles (the caller then uses the packed band solve).
bool tlu_solve(Context& c, const double* rhs, double* z, int accumulate, const int* skip, int* reset) {
  Dev& D = *c.dev;
  if (!D.tlu || !D.tlu->solve_tiles) return false;
  TileLU& L = *D.tlu;
  LAUNCH_NAMED(D, "k_tile_solve", k_tile_solve, kSolveCL, 256, tile_solve_smem(L.NT), c.cs.N0, L.NT, L.TB,
               (const float*)L.T, rhs, z, accumulate, skip, reset, L.solve_status);
  return true;
}

// Raises DeviceTimeout if a cluster solve since the context's setup gave up waiting for its
// partners' rows (synchronises the stream when the tiled solve is in use).
void tlu_check_solves(Context& c) {
  Dev& D = *c.dev;
  if (!D.tlu || !D.tlu->solve_status) return;
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, D.tlu->solve_status, sizeof(int32_t), cudaMemcpyDeviceToHost, D.s));
  CK(cudaStreamSynchronize(D.s));
  if (st == ST_TIMEOUT) throw DeviceTimeout("a CTA of the coarse cluster solve gave up waiting for its partners' rows");
}

}  // namespace nls
