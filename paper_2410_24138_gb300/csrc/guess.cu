// Learned initial guess for the local Newton solves (not part of the paper's method; see
// include/nls.h for the definition of inputs, outputs and the acceptance rule).  Two kinds of
// network: scalar (Eq. 1 on P1 triangles) and displacement (Eq. 2 on Q1 quadrilaterals, two
// components per node).
//
// Kernels:
//   k_guess_features   per subdomain: the 4 x 33 side samples of each component of x on the
//                      box one node beyond the local unknowns (clamped to the mesh); Eq. 1:
//                      log k on 16 x 16 points and the load factor times f; Eq. 2: the load
//                      factor; box width and height (raw values).
//   k_normalise        raw features -> network inputs ((x - mean) / scale).
//   k_gemm_bf16        C = A B with BF16 operands on the tensor cores (mma.sync m16n8k16,
//                      FP32 accumulation); operands are read as FP32 and rounded to BF16 when
//                      staged, so master weights and activations stay FP32.
//   k_gemm_f32         the same product in FP32 (inference and the FP32 gradient check).
//   k_guess_decode     guess at every local unknown = Coons patch of its component's side
//                      samples + bilinear interpolation of that component's 32 x 32 correction.
//   k_guess_harvest    training pair: raw features + correction (w - Coons) of the converged
//                      local state, per component, sampled bilinearly on the canonical grid.
//   k_adam             one Adam step on the FP32 master parameters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "dev_state.cuh"
#include "device.cuh"
#include "nls_internal.h"

namespace nls {

constexpr int kSide = 33, kKS = 16, kGrid = 32;
constexpr int kNF = NLS_GUESS_FEATURES, kNO = NLS_GUESS_OUTPUTS, kG2 = kGrid * kGrid;
constexpr int kNF2 = NLS_GUESS_FEATURES_DISP, kNO2 = NLS_GUESS_OUTPUTS_DISP;
static_assert(4 * kSide + kKS * kKS + 3 == kNF, "feature layout (Eq. 1)");
static_assert(kG2 == kNO, "output layout (Eq. 1)");
static_assert(2 * 4 * kSide + 3 == kNF2, "feature layout (Eq. 2)");
static_assert(2 * kG2 == kNO2, "output layout (Eq. 2)");

// ------------------------------------------------------------------------------------------
// network state
// ------------------------------------------------------------------------------------------
struct GuessNet {
  int device = 0;
  int kind = NLS_GUESS_KIND_SCALAR, nf = kNF, no = kNO;  // inputs and outputs per subdomain
  int h1 = 0, h2 = 0;
  int64_t capacity = 0, npairs = 0, nparam = 0;
  int64_t off[6] = {0};  // W1, b1, W2, b2, W3, b3
  int adam_t = 0;
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  float *mean = nullptr, *scale = nullptr;
  float tscale = 1.f;
  float *dX = nullptr, *dT = nullptr;  // raw dataset
  // work buffers for batches of up to bmax rows
  int bmax = 0;
  float *X = nullptr, *T = nullptr, *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *Y = nullptr;
  float *dA = nullptr, *dZ = nullptr, *lossbuf = nullptr;
  int32_t* idx = nullptr;
  std::vector<void*> allocs;
  template <typename T>
  T* alloc(size_t n) {
    void* q = nullptr;
    CK(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    allocs.push_back(q);
    return (T*)q;
  }
  void ensure_batch(int B);
};

// per-context attachment: geometry maps and buffers
struct GuessCtx {
  GuessNet* net = nullptr;
  int mode = 0;
  int nsub = 0;
  int ndof = 1;  // components per node (the network's kind)
  // per subdomain: side sample maps (node0, node1, weight), k sample elements and f element
  // (Eq. 1), box
  int32_t *side_n0 = nullptr, *side_n1 = nullptr, *kelem = nullptr, *felem = nullptr;
  float *side_w = nullptr, *box = nullptr;  // box: Lx, Ly
  // per local unknown (concatenated as the local states): (s, t) of its node in the box
  double2* st = nullptr;
  // per canonical point of every subdomain: 4 local-unknown positions (-1 = ring) and weights
  int4* cidx = nullptr;
  float2* cw = nullptr;
  // buffers
  float *raw = nullptr, *xin = nullptr, *yout = nullptr;
  double* side = nullptr;  // side samples [nsub][ndof x 132] of the last feature pass
  double* guess = nullptr; // proposed local states (total local unknowns)
  int32_t* accepted = nullptr;
  double* fcell_dev = nullptr;
  double* diag = nullptr;  // per local unknown: the Jacobi smoothing's diagonal
  int sweeps = 6;  // smoothing defaults: 6 sweeps for the scalar kind, 2 for the displacement kind
  double omega = 0.8;
  int64_t proposed_total = 0, accepted_total = 0;
  std::vector<void*> allocs;
  template <typename T>
  T* upload(Dev& D, const std::vector<T>& h) {
    void* q = nullptr;
    CK(cudaMalloc(&q, std::max<size_t>(h.size(), 1) * sizeof(T)));
    allocs.push_back(q);
    if (!h.empty()) CK(cudaMemcpyAsync(q, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, D.s));
    return (T*)q;
  }
  template <typename T>
  T* alloc(size_t n) {
    void* q = nullptr;
    CK(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    allocs.push_back(q);
    return (T*)q;
  }
  ~GuessCtx() {
    for (void* q : allocs) cudaFree(q);
  }
};

namespace {

// ------------------------------------------------------------------------------------------
// splitmix64 on the host (weights and minibatch indices)
// ------------------------------------------------------------------------------------------
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u1 = std::max(uniform(), 1e-300), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
  }
};

// ------------------------------------------------------------------------------------------
// GEMM: C[i, j] = beta C[i, j] + sum_k A(i, k) B(k, j), A(i, k) = A[i sai + k sak],
// B(k, j) = B[k sbk + j sbj]; C row-major with ldc.
// ------------------------------------------------------------------------------------------
__device__ inline uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, int64_t sai,
                                                   int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbj,
                                                   float* __restrict__ C, int64_t ldc, float beta) {
  // 64 x 64 tile, 4 warps in 2 x 2, each warp 32 x 32 = 2 x 4 tiles of 16 x 8
  __shared__ __nv_bfloat16 As[64][16 + 8];
  __shared__ __nv_bfloat16 Bs[64][16 + 8];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int wm = (wid >> 1) * 32, wn = (wid & 1) * 32;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = tid; e < 64 * 16; e += 128) {
      const int r = e / 16, kk = e % 16;
      const int i = i0 + r, k = k0 + kk;
      As[r][kk] = __float2bfloat16_rn((i < M && k < K) ? A[i * sai + k * sak] : 0.f);
      const int j = j0 + r;
      Bs[r][kk] = __float2bfloat16_rn((j < N && k < K) ? B[k * sbk + j * sbj] : 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16;
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&As[r + g][2 * t]);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][2 * t]);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&As[r + g][2 * t + 8]);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][2 * t + 8]);
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int cn = wn + ni * 8;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[cn + g][2 * t]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[cn + g][2 * t + 8]);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + wm + mi * 16 + g + (c >= 2 ? 8 : 0);
        const int j = j0 + wn + ni * 8 + 2 * t + (c & 1);
        if (i < M && j < N) {
          float* cp = C + i * ldc + j;
          *cp = (beta != 0.f ? beta * *cp : 0.f) + acc[mi][ni][c];
        }
      }
}

__global__ void __launch_bounds__(256) k_gemm_f32(int M, int N, int K, const float* __restrict__ A, int64_t sai,
                                                  int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbj,
                                                  float* __restrict__ C, int64_t ldc, float beta) {
  __shared__ float As[16][17], Bs[16][17];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    As[ty][tx] = (blockIdx.y * 16 + ty < M && k0 + tx < K) ? A[(int64_t)(blockIdx.y * 16 + ty) * sai + (k0 + tx) * sak] : 0.f;
    Bs[ty][tx] = (k0 + ty < K && blockIdx.x * 16 + tx < N) ? B[(int64_t)(k0 + ty) * sbk + (blockIdx.x * 16 + tx) * sbj] : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
    __syncthreads();
  }
  if (i < M && j < N) {
    float* cp = C + (int64_t)i * ldc + j;
    *cp = (beta != 0.f ? beta * *cp : 0.f) + acc;
  }
}

void gemm(cudaStream_t s, bool bf16, int M, int N, int K, const float* A, int64_t sai, int64_t sak, const float* B,
          int64_t sbk, int64_t sbj, float* C, int64_t ldc, float beta = 0.f) {
  if (bf16) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, beta);
  } else {
    dim3 grid((N + 15) / 16, (M + 15) / 16);
    k_gemm_f32<<<grid, 256, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, beta);
  }
  CK(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------
// elementwise pieces
// ------------------------------------------------------------------------------------------
__device__ inline float gelu_f(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  return 0.5f * z * (1.f + tanhf(u));
}
__device__ inline float gelu_grad_f(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  const float th = tanhf(u);
  const float du = 0.7978845608028654f * (1.f + 3.f * 0.044715f * z * z);
  return 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * du;
}

// Z += bias (per column); A = gelu(Z) when act != 0
__global__ void k_bias_act(int B, int n, float* Z, const float* bias, float* A, int act) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * n; e += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[e] + bias[e % n];
    Z[e] = z;
    if (act) A[e] = gelu_f(z);
  }
}

// dY = (Y - T) / B; per-block partial losses (fixed order) into part
__global__ void k_loss_grad(int64_t total, int B, const float* Y, const float* T, float* dY, float* part) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = d / (float)B;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0] / (2.f * (float)B);
}

__global__ void k_gelu_back(int64_t total, const float* Z, float* dAZ) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dAZ[e] *= gelu_grad_f(Z[e]);
}

__global__ void k_colsum(int B, int n, const float* dZ, float* db) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int i = 0; i < B; ++i) acc += dZ[(int64_t)i * n + j];
    db[j] = acc;
  }
}

__global__ void k_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// minibatch: X = normalised raw features, T = raw targets / tscale
__global__ void k_gather_batch(int B, int nf, int no, const int32_t* idx, const float* dX, const float* dT,
                               const float* mean, const float* scale, float tscale, float* X, float* T) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * (nf + no);
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / (nf + no)), c = (int)(e % (nf + no));
    const int64_t src = idx[r];
    if (c < nf) X[(int64_t)r * nf + c] = (dX[src * nf + c] - mean[c]) / scale[c];
    else T[(int64_t)r * no + (c - nf)] = dT[src * no + (c - nf)] / tscale;
  }
}

__global__ void k_normalise(int B, int nf, const float* raw, const float* mean, const float* scale, float* X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * nf; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nf);
    X[e] = (raw[e] - mean[c]) / scale[c];
  }
}

// per-feature mean and standard deviation over the first n pairs (fixed-order sums)
__global__ void k_feature_stats(int64_t n, int nf, const float* dX, float* mean, float* scale) {
  const int c = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += dX[r * nf + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double mu = red[0] / (double)n;
  __syncthreads();
  double q = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = dX[r * nf + c] - mu;
    q += d * d;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mean[c] = (float)mu;
    const double sd = sqrt(red[0] / (double)n);
    scale[c] = (float)(sd > 1e-12 ? sd : 1.0);
  }
}

__global__ void k_target_rms(int64_t total, const float* dT, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) s += (double)dT[e] * dT[e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0] / (double)(total > 0 ? total : 1));
}

// ------------------------------------------------------------------------------------------
// geometry kernels (one CTA per subdomain)
// ------------------------------------------------------------------------------------------
struct GeoArgs {
  const SubMeta* meta;
  const int32_t *side_n0, *side_n1, *kelem, *felem;
  const float *side_w, *box;
  const double2* st;
  const int4* cidx;
  const float2* cw;
  const double* kcoef;
  const double* fcell;
  const double* x;
  double load;
  float* raw;
  double* side;
  int ndof, nf;  // components per node, inputs per subdomain
};

__device__ inline double side_value(const double* S, int side, double u) {
  // linear interpolation among the kSide samples of one side, u in [0, 1]
  const double q = u * (kSide - 1);
  int i0 = (int)floor(q);
  i0 = max(0, min(kSide - 2, i0));
  const double w = q - i0;
  return (1.0 - w) * S[side * kSide + i0] + w * S[side * kSide + i0 + 1];
}

__device__ inline double coons_eval(const double* S, double s, double t) {
  // sides: 0 bottom (t = 0), 1 top (t = 1), 2 left (s = 0), 3 right (s = 1)
  const double P00 = S[0], P10 = S[kSide - 1], P01 = S[kSide], P11 = S[2 * kSide - 1];
  return (1 - t) * side_value(S, 0, s) + t * side_value(S, 1, s) + (1 - s) * side_value(S, 2, t) +
         s * side_value(S, 3, t) - ((1 - s) * (1 - t) * P00 + s * (1 - t) * P10 + (1 - s) * t * P01 + s * t * P11);
}

__device__ inline double corr_eval(const float* Y, double s, double t, float tscale) {
  // bilinear interpolation of the kGrid x kGrid correction at (s, t); grid points at (a + 0.5) / kGrid
  double gx = s * kGrid - 0.5, gy = t * kGrid - 0.5;
  gx = fmin(fmax(gx, 0.0), kGrid - 1.0);
  gy = fmin(fmax(gy, 0.0), kGrid - 1.0);
  int a0 = min((int)gx, kGrid - 2), b0 = min((int)gy, kGrid - 2);
  const double wa = gx - a0, wb = gy - b0;
  const double v = (1 - wa) * (1 - wb) * Y[b0 * kGrid + a0] + wa * (1 - wb) * Y[b0 * kGrid + a0 + 1] +
                   (1 - wa) * wb * Y[(b0 + 1) * kGrid + a0] + wa * wb * Y[(b0 + 1) * kGrid + a0 + 1];
  return v * tscale;
}

// Eq. 1: [side samples (132), log k (256), load f, box width, box height]; Eq. 2: [side samples of
// component 0 (132), of component 1 (132), load, box width, box height].
__global__ void k_guess_features(GeoArgs G, int nsub) {
  const int sub = blockIdx.x;
  if (sub >= nsub) return;
  constexpr int NS = 4 * kSide;
  const int nd = G.ndof;
  float* out = G.raw + (int64_t)sub * G.nf;
  double* S = G.side + (int64_t)sub * nd * NS;
  for (int e = threadIdx.x; e < nd * NS; e += blockDim.x) {
    const int c = e / NS, q = e % NS;
    const int64_t k = (int64_t)sub * NS + q;
    const double w = G.side_w[k];
    const double v = (1.0 - w) * G.x[(int64_t)G.side_n0[k] * nd + c] + w * G.x[(int64_t)G.side_n1[k] * nd + c];
    S[e] = v;
    out[e] = (float)v;
  }
  if (nd == 1) {
    for (int q = threadIdx.x; q < kKS * kKS; q += blockDim.x)
      out[NS + q] = (float)log(G.kcoef[G.kelem[(int64_t)sub * kKS * kKS + q]]);
    if (threadIdx.x == 0) {
      out[NS + kKS * kKS] = (float)(G.load * G.fcell[G.felem[sub]]);
      out[NS + kKS * kKS + 1] = G.box[2 * sub];
      out[NS + kKS * kKS + 2] = G.box[2 * sub + 1];
    }
  } else if (threadIdx.x == 0) {
    out[nd * NS] = (float)G.load;
    out[nd * NS + 1] = G.box[2 * sub];
    out[nd * NS + 2] = G.box[2 * sub + 1];
  }
}

// local unknown a is component a % ndof of its node (node-major, component-interleaved)
__global__ void k_guess_decode(GeoArgs G, int nsub, const float* Y, float tscale, double* guess) {
  const int sub = blockIdx.x;
  if (sub >= nsub) return;
  const SubMeta m = G.meta[sub];
  const int nd = G.ndof;
  const double* S = G.side + (int64_t)sub * nd * 4 * kSide;
  const float* Ys = Y + (int64_t)sub * nd * kG2;
  for (int a = threadIdx.x; a < m.n; a += blockDim.x) {
    const int c = a % nd;
    const double2 p = G.st[m.vec_off + a];
    guess[m.vec_off + a] = coons_eval(S + c * 4 * kSide, p.x, p.y) + corr_eval(Ys + c * kG2, p.x, p.y, tscale);
  }
}

// Harvest: raw features (already in G.raw) and the correction of the converged local state w
// sampled on the canonical grid.
__global__ void k_guess_harvest(GeoArgs G, int nsub, const double* w, float* dX, float* dT, int64_t slot0) {
  const int sub = blockIdx.x;
  if (sub >= nsub) return;
  const SubMeta m = G.meta[sub];
  const int nd = G.ndof;
  const double* S = G.side + (int64_t)sub * nd * 4 * kSide;
  float* X = dX + (slot0 + sub) * G.nf;
  float* T = dT + (slot0 + sub) * nd * kG2;
  for (int q = threadIdx.x; q < G.nf; q += blockDim.x) X[q] = G.raw[(int64_t)sub * G.nf + q];
  for (int e = threadIdx.x; e < nd * kG2; e += blockDim.x) {
    const int comp = e / kG2, q = e % kG2;
    const int4 id = G.cidx[(int64_t)sub * kG2 + q];
    const float2 wt = G.cw[(int64_t)sub * kG2 + q];
    const int ids[4] = {id.x, id.y, id.z, id.w};
    const double wts[4] = {(1.0 - wt.x) * (1.0 - wt.y), wt.x * (1.0 - wt.y), (1.0 - wt.x) * wt.y, wt.x * wt.y};
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (ids[c] >= 0) {
        const int64_t l = m.vec_off + (int64_t)ids[c] * nd + comp;
        const double2 p = G.st[l];
        v += wts[c] * (w[l] - coons_eval(S + comp * 4 * kSide, p.x, p.y));
      }
    T[e] = (float)v;
  }
}

}  // namespace

void GuessNet::ensure_batch(int B) {
  if (B <= bmax) return;
  bmax = B;
  X = alloc<float>((size_t)B * nf);
  T = alloc<float>((size_t)B * no);
  const int hm = std::max(h1, h2);
  Z1 = alloc<float>((size_t)B * h1);
  A1 = alloc<float>((size_t)B * h1);
  Z2 = alloc<float>((size_t)B * h2);
  A2 = alloc<float>((size_t)B * h2);
  Y = alloc<float>((size_t)B * no);
  dA = alloc<float>((size_t)B * std::max(hm, no));
  dZ = alloc<float>((size_t)B * std::max(hm, no));
  lossbuf = alloc<float>(1024);
  idx = alloc<int32_t>(B);
}

namespace {

// forward pass of B rows of normalised inputs in net.X (or `X` if given) into net.Y
void net_forward(GuessNet& N, cudaStream_t s, int B, const float* X, bool bf16) {
  const float* W1 = N.p + N.off[0];
  const float* b1 = N.p + N.off[1];
  const float* W2 = N.p + N.off[2];
  const float* b2 = N.p + N.off[3];
  const float* W3 = N.p + N.off[4];
  const float* b3 = N.p + N.off[5];
  const int grid = 1216;
  gemm(s, bf16, B, N.h1, N.nf, X, N.nf, 1, W1, 1, N.nf, N.Z1, N.h1);
  k_bias_act<<<grid, 256, 0, s>>>(B, N.h1, N.Z1, b1, N.A1, 1);
  gemm(s, bf16, B, N.h2, N.h1, N.A1, N.h1, 1, W2, 1, N.h1, N.Z2, N.h2);
  k_bias_act<<<grid, 256, 0, s>>>(B, N.h2, N.Z2, b2, N.A2, 1);
  gemm(s, bf16, B, N.no, N.h2, N.A2, N.h2, 1, W3, 1, N.h2, N.Y, N.no);
  k_bias_act<<<grid, 256, 0, s>>>(B, N.no, N.Y, b3, nullptr, 0);
  CK(cudaGetLastError());
}

// loss and gradient (into N.g) of the batch in N.X / N.T
float net_gradient(GuessNet& N, cudaStream_t s, int B, bool bf16) {
  net_forward(N, s, B, N.X, bf16);
  const float* W2 = N.p + N.off[2];
  const float* W3 = N.p + N.off[4];
  const int nb = 256;
  k_loss_grad<<<nb, 256, 0, s>>>((int64_t)B * N.no, B, N.Y, N.T, N.dZ, N.lossbuf);
  // layer 3: dW3 = dY^T A2, db3 = colsum dY, dA2 = dY W3
  gemm(s, bf16, N.no, N.h2, B, N.dZ, 1, N.no, N.A2, N.h2, 1, N.g + N.off[4], N.h2);
  k_colsum<<<(N.no + 255) / 256, 256, 0, s>>>(B, N.no, N.dZ, N.g + N.off[5]);
  gemm(s, bf16, B, N.h2, N.no, N.dZ, N.no, 1, W3, N.h2, 1, N.dA, N.h2);
  k_gelu_back<<<1216, 256, 0, s>>>((int64_t)B * N.h2, N.Z2, N.dA);
  // layer 2 (dZ2 in dA)
  gemm(s, bf16, N.h2, N.h1, B, N.dA, 1, N.h2, N.A1, N.h1, 1, N.g + N.off[2], N.h1);
  k_colsum<<<(N.h2 + 255) / 256, 256, 0, s>>>(B, N.h2, N.dA, N.g + N.off[3]);
  gemm(s, bf16, B, N.h1, N.h2, N.dA, N.h2, 1, W2, N.h1, 1, N.dZ, N.h1);
  k_gelu_back<<<1216, 256, 0, s>>>((int64_t)B * N.h1, N.Z1, N.dZ);
  // layer 1 (dZ1 in dZ)
  gemm(s, bf16, N.h1, N.nf, B, N.dZ, 1, N.h1, N.X, N.nf, 1, N.g + N.off[0], N.nf);
  k_colsum<<<(N.h1 + 255) / 256, 256, 0, s>>>(B, N.h1, N.dZ, N.g + N.off[1]);
  CK(cudaGetLastError());
  std::vector<float> part(nb);
  CK(cudaMemcpyAsync(part.data(), N.lossbuf, nb * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double L = 0.0;
  for (float v : part) L += v;
  return (float)L;
}

// ------------------------------------------------------------------------------------------
// host geometry of the attachment (structured P1 or Q1 meshes of the unit square)
// ------------------------------------------------------------------------------------------
// Leading-term Jacobian diagonal of every local unknown: sum over the subdomain's elements of
// k_e |grad phi_a|^2 |e| (the smoothing of proposed starts divides by it times (1 + w_a^2)).
std::vector<double> jacobi_diagonal(const Context& c) {
  const LocalSet& s = c.ov;
  std::vector<double> diag(s.total_n, 0.0);
  for (int sb = 0; sb < s.count; ++sb) {
    const SubMeta& m = s.meta[sb];
    for (int e = 0; e < m.ne; ++e) {
      const int64_t ge = s.elem_gid[m.elem_off + e];
      const double* g = &c.geom[ge * c.geom_stride];
      const double ke = c.k_elem.empty() ? 1.0 : c.k_elem[ge];
      for (int a = 0; a < 3; ++a) {
        const int t = s.lconn[(m.elem_off + e) * 3 + a];
        if (t < m.n) diag[m.vec_off + t] += ke * g[6] * (g[2 * a] * g[2 * a] + g[2 * a + 1] * g[2 * a + 1]);
      }
    }
    for (int a = 0; a < m.n; ++a)
      if (!(diag[m.vec_off + a] > 0.0)) throw std::runtime_error("learned guess: zero Jacobi diagonal");
  }
  return diag;
}

// Eq. 2: diagonal of the linear-elastic Q1 stiffness (the tangent at zero displacement) at every
// local unknown, sum over elements and Gauss points of w det(J) ((lambda + 2 mu) (dN_a/dX_c)^2 +
// mu (dN_a/dX_c')^2) for component c (c' the other one).
std::vector<double> elasticity_diagonal(const Context& c) {
  const LocalSet& s = c.ov;
  double mu = 0.0, lam = 0.0;
  lame(c, mu, lam);
  std::vector<double> diag(s.total_n, 0.0);
  for (int sb = 0; sb < s.count; ++sb) {
    const SubMeta& m = s.meta[sb];
    for (int e = 0; e < m.ne; ++e) {
      const int64_t ge = s.elem_gid[m.elem_off + e];
      for (int q = 0; q < 4; ++q) {
        const double* g = &c.geom[ge * c.geom_stride + q * 10];
        for (int a = 0; a < 4; ++a) {
          const int t = s.lconn[(m.elem_off + e) * 4 + a];
          if (t >= m.nV) continue;
          const double gx = g[2 * a], gy = g[2 * a + 1];
          diag[m.vec_off + 2 * t] += g[8] * ((lam + 2.0 * mu) * gx * gx + mu * gy * gy);
          diag[m.vec_off + 2 * t + 1] += g[8] * ((lam + 2.0 * mu) * gy * gy + mu * gx * gx);
        }
      }
    }
    for (int a = 0; a < m.n; ++a)
      if (!(diag[m.vec_off + a] > 0.0)) throw std::runtime_error("learned guess: zero Jacobi diagonal");
  }
  return diag;
}

// The scalar kind needs Eq. 1 on P1 triangles, the displacement kind Eq. 2 on Q1 quadrilaterals.
bool guess_kind_matches(const Context& c, int kind) {
  if (kind == NLS_GUESS_KIND_SCALAR) return c.elem_type == NLS_P1_TRI && c.ndof == 1;
  return kind == NLS_GUESS_KIND_DISPLACEMENT && c.elem_type == NLS_Q1_QUAD && c.ndof == 2 &&
         c.law == NLS_LAW_NEOHOOKE;
}

void build_geometry(Context& c, GuessCtx& G) {
  const int nd = c.ndof;
  G.ndof = nd;
  // grid indices from coordinates
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    xmin = std::min(xmin, c.xy[2 * v]);
    xmax = std::max(xmax, c.xy[2 * v]);
    ymin = std::min(ymin, c.xy[2 * v + 1]);
    ymax = std::max(ymax, c.xy[2 * v + 1]);
  }
  const int64_t side = (int64_t)std::llround(std::sqrt((double)c.n_nodes));
  if (side * side != c.n_nodes) throw std::runtime_error("learned guess: mesh is not a square structured grid");
  const int nn = (int)side - 1;  // cells per side
  const double hx = (xmax - xmin) / nn, hy = (ymax - ymin) / nn;
  std::vector<int32_t> gi(c.n_nodes), gj(c.n_nodes);
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    const double fx = (c.xy[2 * v] - xmin) / hx, fy = (c.xy[2 * v + 1] - ymin) / hy;
    gi[v] = (int32_t)std::llround(fx);
    gj[v] = (int32_t)std::llround(fy);
    if (std::abs(fx - gi[v]) > 1e-6 || std::abs(fy - gj[v]) > 1e-6 || gj[v] * side + gi[v] != v)
      throw std::runtime_error("learned guess: nodes are not numbered as a lexicographic structured grid");
  }
  auto node = [&](int i, int j) { return (int32_t)(j * side + i); };
  const LocalSet& s = c.ov;
  const int nsub = s.count;
  const bool scalar = nd == 1;
  std::vector<int32_t> n0((size_t)nsub * 4 * kSide), n1((size_t)nsub * 4 * kSide),
      kel(scalar ? (size_t)nsub * kKS * kKS : 0), fel(scalar ? nsub : 0);
  std::vector<float> sw((size_t)nsub * 4 * kSide), box(2 * (size_t)nsub);
  std::vector<double2> st(s.total_n);
  const std::vector<double> diag = scalar ? jacobi_diagonal(c) : elasticity_diagonal(c);
  std::vector<int4> cidx((size_t)nsub * kG2);
  std::vector<float2> cw((size_t)nsub * kG2);
  for (int sb = 0; sb < nsub; ++sb) {
    const SubMeta& m = s.meta[sb];
    int ia = INT32_MAX, ib = -1, ja = INT32_MAX, jb = -1;
    std::map<int64_t, int> local;  // node -> local unknown index
    for (int a = 0; a < m.nV; ++a) {
      const int32_t v = s.tnode_gid[m.tnode_off + a];
      ia = std::min(ia, gi[v]);
      ib = std::max(ib, gi[v]);
      ja = std::min(ja, gj[v]);
      jb = std::max(jb, gj[v]);
      local[v] = a;
    }
    // box [ia-1, ib+1] x [ja-1, jb+1] clamped to the mesh (the clamp acts only where local
    // unknowns reach a Neumann edge)
    const int i0 = std::max(ia - 1, 0), i1 = std::min(ib + 1, nn), j0 = std::max(ja - 1, 0), j1 = std::min(jb + 1, nn);
    const double Lx = (i1 - i0) * hx, Ly = (j1 - j0) * hy;
    box[2 * sb] = (float)Lx;
    box[2 * sb + 1] = (float)Ly;
    for (int q = 0; q < kSide; ++q) {
      const double u = (double)q / (kSide - 1);
      // bottom / top: along i at j0 / j1; left / right: along j at i0 / i1
      const double fi = i0 + u * (i1 - i0), fj = j0 + u * (j1 - j0);
      int ii = std::min((int)std::floor(fi), i1 - 1), jj = std::min((int)std::floor(fj), j1 - 1);
      const double wi = fi - ii, wj = fj - jj;
      const size_t base = (size_t)sb * 4 * kSide;
      n0[base + q] = node(ii, j0);
      n1[base + q] = node(ii + 1, j0);
      sw[base + q] = (float)wi;
      n0[base + kSide + q] = node(ii, j1);
      n1[base + kSide + q] = node(ii + 1, j1);
      sw[base + kSide + q] = (float)wi;
      n0[base + 2 * kSide + q] = node(i0, jj);
      n1[base + 2 * kSide + q] = node(i0, jj + 1);
      sw[base + 2 * kSide + q] = (float)wj;
      n0[base + 3 * kSide + q] = node(i1, jj);
      n1[base + 3 * kSide + q] = node(i1, jj + 1);
      sw[base + 3 * kSide + q] = (float)wj;
    }
    for (int b = 0; b < (scalar ? kKS : 0); ++b)
      for (int a = 0; a < kKS; ++a) {
        const double fx = i0 + (a + 0.5) / kKS * (i1 - i0), fy = j0 + (b + 0.5) / kKS * (j1 - j0);
        const int ci = std::min((int)fx, nn - 1), cj = std::min((int)fy, nn - 1);
        // SW-NE diagonal: the lower triangle (2c) when the point is below the diagonal
        const bool lower = (fx - ci) >= (fy - cj);
        kel[(size_t)sb * kKS * kKS + b * kKS + a] = 2 * (cj * nn + ci) + (lower ? 0 : 1);
      }
    if (scalar) {
      const int ci = std::min((i0 + i1) / 2, nn - 1), cj = std::min((j0 + j1) / 2, nn - 1);
      fel[sb] = 2 * (cj * nn + ci);
    }
    for (int a = 0; a < m.n; ++a) {
      const int32_t v = s.tnode_gid[m.tnode_off + a / nd];
      st[m.vec_off + a] = make_double2((gi[v] - i0) / (double)(i1 - i0), (gj[v] - j0) / (double)(j1 - j0));
    }
    for (int b = 0; b < kGrid; ++b)
      for (int a = 0; a < kGrid; ++a) {
        const double fx = i0 + (a + 0.5) / kGrid * (i1 - i0), fy = j0 + (b + 0.5) / kGrid * (j1 - j0);
        const int ii = std::min((int)std::floor(fx), i1 - 1), jj = std::min((int)std::floor(fy), j1 - 1);
        auto lid = [&](int i, int j) {
          auto it = local.find(node(i, j));
          return it == local.end() ? -1 : it->second;
        };
        cidx[(size_t)sb * kG2 + b * kGrid + a] = make_int4(lid(ii, jj), lid(ii + 1, jj), lid(ii, jj + 1), lid(ii + 1, jj + 1));
        cw[(size_t)sb * kG2 + b * kGrid + a] = make_float2((float)(fx - ii), (float)(fy - jj));
      }
  }
  Dev& D = *c.dev;
  G.nsub = nsub;
  G.side_n0 = G.upload(D, n0);
  G.side_n1 = G.upload(D, n1);
  G.side_w = G.upload(D, sw);
  G.kelem = G.upload(D, kel);
  G.felem = G.upload(D, fel);
  G.box = G.upload(D, box);
  G.st = G.upload(D, st);
  G.cidx = G.upload(D, cidx);
  G.cw = G.upload(D, cw);
  G.diag = G.upload(D, diag);
  G.raw = G.alloc<float>((size_t)nsub * G.net->nf);
  G.xin = G.alloc<float>((size_t)nsub * G.net->nf);
  G.side = G.alloc<double>((size_t)nsub * nd * 4 * kSide);
  G.guess = G.alloc<double>(s.total_n);
  G.accepted = G.alloc<int32_t>(nsub);
  std::vector<double> fcell(c.n_elems, 1.0);
  if (!c.f_elem.empty()) fcell = c.f_elem;
  G.fcell_dev = G.upload(D, fcell);
  CK(cudaStreamSynchronize(D.s));
}

GeoArgs geo_args(Context& c, GuessCtx& G, const double* x, double load) {
  GeoArgs a;
  std::memset(&a, 0, sizeof(a));
  Dev& D = *c.dev;
  a.meta = D.ov.meta;
  a.side_n0 = G.side_n0;
  a.side_n1 = G.side_n1;
  a.kelem = G.kelem;
  a.felem = G.felem;
  a.side_w = G.side_w;
  a.box = G.box;
  a.st = G.st;
  a.cidx = G.cidx;
  a.cw = G.cw;
  a.kcoef = D.kcoef;
  a.fcell = G.fcell_dev;
  a.x = x;
  a.load = load;
  a.raw = G.raw;
  a.side = G.side;
  a.ndof = G.ndof;
  a.nf = G.net->nf;
  return a;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// hooks used by the solver
// ------------------------------------------------------------------------------------------
GuessProposal guess_propose(Context& c, const double* x, double load) {
  Dev& D = *c.dev;
  GuessCtx* G = (GuessCtx*)D.guess;
  GuessProposal out;
  if (!G || !(G->mode & NLS_GUESS_USE) || !G->net) return out;
  if ((G->mode & NLS_GUESS_FIRST_OUTER) && D.outer_k > 0) return out;
  GuessNet& N = *G->net;
  N.ensure_batch(G->nsub);
  GeoArgs a = geo_args(c, *G, x, load);
  LAUNCH(D, k_guess_features, G->nsub, 128, 0, a, G->nsub);
  LAUNCH(D, k_normalise, 1216, 256, 0, G->nsub, N.nf, G->raw, N.mean, N.scale, G->xin);
  net_forward(N, D.s, G->nsub, G->xin, false);
  D.launches += 6;
  LAUNCH(D, k_guess_decode, G->nsub, 128, 0, a, G->nsub, N.Y, N.tscale, G->guess);
  CK(cudaMemsetAsync(G->accepted, 0, sizeof(int32_t) * G->nsub, D.s));
  G->proposed_total += G->nsub;
  out.x = G->guess;
  out.accepted = G->accepted;
  out.diag = G->diag;
  out.sweeps = G->sweeps;
  out.omega = G->omega;
  return out;
}

// Smoothing parameters of the attached guess (diagonal, sweeps, omega) without a proposal.
GuessProposal guess_smoothing(Context& c) {
  GuessProposal out;
  GuessCtx* G = c.dev ? (GuessCtx*)c.dev->guess : nullptr;
  if (!G) return out;
  out.diag = G->diag;
  out.sweeps = G->sweeps;
  out.omega = G->omega;
  return out;
}

// Test hooks: the raw features at x (host) into out [nsub x nf], and the decode of given network
// outputs Y [nsub x no] (normalised units) at x into out [total local unknowns].
int guess_features(Context& c, const double* x, double load, float* out) {
  GuessCtx* G = c.dev ? (GuessCtx*)c.dev->guess : nullptr;
  if (!G) {
    c.last_error = "the learned-guess hooks need an attached network";
    return NLS_E_ARG;
  }
  Dev& D = *c.dev;
  try {
    CK(cudaMemcpyAsync(D.x, x, sizeof(double) * c.N, cudaMemcpyHostToDevice, D.s));
    GeoArgs a = geo_args(c, *G, D.x, load);
    LAUNCH(D, k_guess_features, G->nsub, 128, 0, a, G->nsub);
    CK(cudaMemcpyAsync(out, G->raw, sizeof(float) * (size_t)G->nsub * G->net->nf, cudaMemcpyDeviceToHost, D.s));
    CK(cudaStreamSynchronize(D.s));
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int guess_decode(Context& c, const double* x, double load, const float* Y, double* out) {
  GuessCtx* G = c.dev ? (GuessCtx*)c.dev->guess : nullptr;
  if (!G || !G->net) {
    c.last_error = "the learned-guess hooks need an attached network";
    return NLS_E_ARG;
  }
  Dev& D = *c.dev;
  GuessNet& N = *G->net;
  try {
    N.ensure_batch(G->nsub);
    CK(cudaMemcpyAsync(D.x, x, sizeof(double) * c.N, cudaMemcpyHostToDevice, D.s));
    CK(cudaMemcpyAsync(N.Y, Y, sizeof(float) * (size_t)G->nsub * N.no, cudaMemcpyHostToDevice, D.s));
    GeoArgs a = geo_args(c, *G, D.x, load);
    LAUNCH(D, k_guess_features, G->nsub, 128, 0, a, G->nsub);
    LAUNCH(D, k_guess_decode, G->nsub, 128, 0, a, G->nsub, N.Y, N.tscale, G->guess);
    CK(cudaMemcpyAsync(out, G->guess, sizeof(double) * c.ov.total_n, cudaMemcpyDeviceToHost, D.s));
    CK(cudaStreamSynchronize(D.s));
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int guess_set_smoothing(Context& c, int32_t sweeps, double omega) {
  GuessCtx* G = c.dev ? (GuessCtx*)c.dev->guess : nullptr;
  if (!G) {
    c.last_error = "nls_guess_set_smoothing needs an attached network";
    return NLS_E_ARG;
  }
  if (sweeps < 0 || sweeps > 64 || !(omega > 0.0 && omega <= 1.0)) {
    c.last_error = "smoothing needs sweeps in [0, 64] and omega in (0, 1]";
    return NLS_E_ARG;
  }
  G->sweeps = sweeps;
  G->omega = omega;
  return NLS_OK;
}

void guess_after_local(Context& c, const double* x, double load, bool proposed) {
  Dev& D = *c.dev;
  GuessCtx* G = (GuessCtx*)D.guess;
  if (!G) return;
  if (proposed) {
    std::vector<int32_t> acc(G->nsub);
    CK(cudaMemcpyAsync(acc.data(), G->accepted, sizeof(int32_t) * G->nsub, cudaMemcpyDeviceToHost, D.s));
    CK(cudaStreamSynchronize(D.s));
    for (int32_t v : acc) G->accepted_total += v;
  }
  if ((G->mode & NLS_GUESS_HARVEST) && G->net) {
    GuessNet& N = *G->net;
    if (N.npairs + G->nsub > N.capacity) return;  // dataset full: stop recording
    GeoArgs a = geo_args(c, *G, x, load);
    if (!proposed) LAUNCH(D, k_guess_features, G->nsub, 128, 0, a, G->nsub);
    LAUNCH(D, k_guess_harvest, G->nsub, 128, 0, a, G->nsub, D.ov.w, N.dX, N.dT, N.npairs);
    N.npairs += G->nsub;
  }
}

// New k / f on an attached context: the per-element f copy and the Jacobi diagonal follow.
void guess_coefficients_changed(Context& c) {
  GuessCtx* G = (c.dev && c.dev->guess) ? (GuessCtx*)c.dev->guess : nullptr;
  if (!G) return;
  Dev& D = *c.dev;
  const std::vector<double> diag = jacobi_diagonal(c);
  CK(cudaMemcpyAsync(G->diag, diag.data(), sizeof(double) * diag.size(), cudaMemcpyHostToDevice, D.s));
  std::vector<double> fcell(c.n_elems, 1.0);
  if (!c.f_elem.empty()) fcell = c.f_elem;
  CK(cudaMemcpyAsync(G->fcell_dev, fcell.data(), sizeof(double) * fcell.size(), cudaMemcpyHostToDevice, D.s));
  CK(cudaStreamSynchronize(D.s));
}

void guess_free(Context& c) {
  if (c.dev && c.dev->guess) {
    delete (GuessCtx*)c.dev->guess;
    c.dev->guess = nullptr;
  }
}

}  // namespace nls

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
using nls::GuessNet;

struct nls_guess_net {
  GuessNet n;
};

extern "C" {

int nls_guess_create(nls_guess_net** out, int device, int32_t h1, int32_t h2, uint64_t seed, int64_t capacity) {
  return nls_guess_create_kind(out, device, NLS_GUESS_KIND_SCALAR, h1, h2, seed, capacity);
}

int nls_guess_create_kind(nls_guess_net** out, int device, int32_t kind, int32_t h1, int32_t h2, uint64_t seed,
                          int64_t capacity) {
  if (!out || h1 <= 0 || h2 <= 0 || h1 % 16 || h2 % 16 || capacity < 0) return NLS_E_ARG;
  if (kind != NLS_GUESS_KIND_SCALAR && kind != NLS_GUESS_KIND_DISPLACEMENT) return NLS_E_ARG;
  nls_guess_net* w = new (std::nothrow) nls_guess_net();
  if (!w) return NLS_E_NOMEM;
  GuessNet& N = w->n;
  try {
    CK(cudaSetDevice(device));
    N.device = device;
    N.kind = kind;
    N.nf = kind == NLS_GUESS_KIND_SCALAR ? nls::kNF : nls::kNF2;
    N.no = kind == NLS_GUESS_KIND_SCALAR ? nls::kNO : nls::kNO2;
    N.h1 = h1;
    N.h2 = h2;
    N.capacity = capacity;
    const int64_t sz[6] = {(int64_t)h1 * N.nf, h1, (int64_t)h2 * h1, h2, (int64_t)N.no * h2, N.no};
    int64_t o = 0;
    for (int k = 0; k < 6; ++k) {
      N.off[k] = o;
      o += sz[k];
    }
    N.nparam = o;
    std::vector<float> p(o, 0.f);
    nls::SplitMix rng{seed};
    const int fan_in[3] = {N.nf, h1, h2};
    for (int l = 0; l < 3; ++l) {
      const double sd = 1.0 / std::sqrt((double)fan_in[l]);
      for (int64_t e = 0; e < sz[2 * l]; ++e) p[N.off[2 * l] + e] = (float)(sd * rng.normal());
    }
    N.p = N.alloc<float>(o);
    N.m = N.alloc<float>(o);
    N.v = N.alloc<float>(o);
    N.g = N.alloc<float>(o);
    CK(cudaMemcpy(N.p, p.data(), o * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemset(N.m, 0, o * sizeof(float)));
    CK(cudaMemset(N.v, 0, o * sizeof(float)));
    N.mean = N.alloc<float>(N.nf);
    N.scale = N.alloc<float>(N.nf);
    std::vector<float> zero(N.nf, 0.f), one(N.nf, 1.f);
    CK(cudaMemcpy(N.mean, zero.data(), N.nf * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(N.scale, one.data(), N.nf * sizeof(float), cudaMemcpyHostToDevice));
    N.dX = N.alloc<float>((size_t)capacity * N.nf);
    N.dT = N.alloc<float>((size_t)capacity * N.no);
  } catch (const std::exception&) {
    for (void* q : N.allocs) cudaFree(q);
    delete w;
    return NLS_E_CUDA;
  }
  *out = w;
  return NLS_OK;
}

void nls_guess_destroy(nls_guess_net* w) {
  if (!w) return;
  cudaSetDevice(w->n.device);
  cudaDeviceSynchronize();
  for (void* q : w->n.allocs) cudaFree(q);
  delete w;
}

int nls_guess_dims(const nls_guess_net* w, int32_t* kind, int32_t* n_in, int32_t* n_out) {
  if (!w) return NLS_E_ARG;
  if (kind) *kind = w->n.kind;
  if (n_in) *n_in = w->n.nf;
  if (n_out) *n_out = w->n.no;
  return NLS_OK;
}

int nls_guess_pairs(const nls_guess_net* w, int64_t* n) {
  if (!w || !n) return NLS_E_ARG;
  *n = w->n.npairs;
  return NLS_OK;
}

int nls_guess_get_params(const nls_guess_net* w, float* params, int64_t* count) {
  if (!w || !count) return NLS_E_ARG;
  *count = w->n.nparam;
  if (!params) return NLS_OK;
  if (cudaSetDevice(w->n.device) != cudaSuccess) return NLS_E_CUDA;
  return cudaMemcpy(params, w->n.p, w->n.nparam * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? NLS_OK
                                                                                                        : NLS_E_CUDA;
}

int nls_guess_set_params(nls_guess_net* w, const float* params, int64_t count) {
  if (!w || !params || count != w->n.nparam) return NLS_E_ARG;
  GuessNet& N = w->n;
  if (cudaSetDevice(N.device) != cudaSuccess) return NLS_E_CUDA;
  if (cudaMemcpy(N.p, params, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return NLS_E_CUDA;
  cudaMemset(N.m, 0, count * sizeof(float));
  cudaMemset(N.v, 0, count * sizeof(float));
  N.adam_t = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? NLS_OK : NLS_E_CUDA;
}

int nls_guess_get_normalisation(const nls_guess_net* w, float* mean, float* scale, float* tscale) {
  if (!w) return NLS_E_ARG;
  const GuessNet& N = w->n;
  if (cudaSetDevice(N.device) != cudaSuccess) return NLS_E_CUDA;
  if (mean) cudaMemcpy(mean, N.mean, N.nf * sizeof(float), cudaMemcpyDeviceToHost);
  if (scale) cudaMemcpy(scale, N.scale, N.nf * sizeof(float), cudaMemcpyDeviceToHost);
  if (tscale) *tscale = N.tscale;
  return cudaDeviceSynchronize() == cudaSuccess ? NLS_OK : NLS_E_CUDA;
}

int nls_guess_set_normalisation(nls_guess_net* w, const float* mean, const float* scale, float tscale) {
  if (!w || !mean || !scale || !(tscale > 0.f)) return NLS_E_ARG;
  GuessNet& N = w->n;
  if (cudaSetDevice(N.device) != cudaSuccess) return NLS_E_CUDA;
  cudaMemcpy(N.mean, mean, N.nf * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(N.scale, scale, N.nf * sizeof(float), cudaMemcpyHostToDevice);
  N.tscale = tscale;
  return cudaDeviceSynchronize() == cudaSuccess ? NLS_OK : NLS_E_CUDA;
}

int nls_guess_gradient(nls_guess_net* w, int32_t B, const float* X, const float* T, int32_t precision, float* grad,
                       float* loss) {
  if (!w || B <= 0 || !X || !T || !grad) return NLS_E_ARG;
  GuessNet& N = w->n;
  try {
    CK(cudaSetDevice(N.device));
    N.ensure_batch(B);
    CK(cudaMemcpy(N.X, X, (size_t)B * N.nf * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(N.T, T, (size_t)B * N.no * sizeof(float), cudaMemcpyHostToDevice));
    const float L = nls::net_gradient(N, 0, B, precision == 1);
    CK(cudaMemcpy(grad, N.g, N.nparam * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) *loss = L;
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int nls_guess_forward(nls_guess_net* w, int32_t B, const float* X, float* Y) {
  if (!w || B <= 0 || !X || !Y) return NLS_E_ARG;
  GuessNet& N = w->n;
  try {
    CK(cudaSetDevice(N.device));
    N.ensure_batch(B);
    CK(cudaMemcpy(N.X, X, (size_t)B * N.nf * sizeof(float), cudaMemcpyHostToDevice));
    nls::net_forward(N, 0, B, N.X, false);
    CK(cudaMemcpy(Y, N.Y, (size_t)B * N.no * sizeof(float), cudaMemcpyDeviceToHost));
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int nls_guess_train(nls_guess_net* w, int32_t steps, int32_t batch, double lr, uint64_t seed, float* loss_out) {
  if (!w || steps < 0 || batch <= 0) return NLS_E_ARG;
  GuessNet& N = w->n;
  if (N.npairs <= 0) return NLS_E_ARG;
  try {
    CK(cudaSetDevice(N.device));
    N.ensure_batch(batch);
    // normalisation from the harvested pairs (inputs per feature, targets by their rms)
    nls::k_feature_stats<<<N.nf, 256>>>(N.npairs, N.nf, N.dX, N.mean, N.scale);
    double* rms = nullptr;
    CK(cudaMalloc(&rms, sizeof(double)));
    nls::k_target_rms<<<1, 256>>>(N.npairs * N.no, N.dT, rms);
    double hr = 1.0;
    CK(cudaMemcpy(&hr, rms, sizeof(double), cudaMemcpyDeviceToHost));
    cudaFree(rms);
    N.tscale = (float)(hr > 1e-30 ? hr : 1.0);
    nls::SplitMix rng{seed};
    std::vector<int32_t> idx(batch);
    for (int st = 0; st < steps; ++st) {
      for (int r = 0; r < batch; ++r) idx[r] = (int32_t)(rng.next() % (uint64_t)N.npairs);
      CK(cudaMemcpy(N.idx, idx.data(), batch * sizeof(int32_t), cudaMemcpyHostToDevice));
      nls::k_gather_batch<<<1216, 256>>>(batch, N.nf, N.no, N.idx, N.dX, N.dT, N.mean, N.scale, N.tscale, N.X, N.T);
      const float L = nls::net_gradient(N, 0, batch, true);
      N.adam_t += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      nls::k_adam<<<1216, 256>>>(N.nparam, N.p, N.g, N.m, N.v, (float)lr, b1, b2, 1e-8f,
                                 1.f - std::pow(b1, (float)N.adam_t), 1.f - std::pow(b2, (float)N.adam_t));
      CK(cudaGetLastError());
      if (loss_out) loss_out[st] = L;
    }
    CK(cudaDeviceSynchronize());
  } catch (const std::exception&) {
    return NLS_E_CUDA;
  }
  return NLS_OK;
}

int nls_guess_attach(nls_ctx* ctx, nls_guess_net* w, int32_t mode);  // defined in api.cpp (needs the context)

}  // extern "C"

namespace nls {

int guess_attach(Context& c, nls_guess_net* w, int32_t mode) {
  if (!c.is_setup || !c.dev) {
    c.last_error = "nls_guess_attach needs a context after nls_setup";
    return NLS_E_ARG;
  }
  try {
    CK(cudaSetDevice(c.device));
    guess_free(c);
    if (!w || mode == 0) return NLS_OK;
    if (w->n.device != c.device) {
      c.last_error = "network and context live on different devices";
      return NLS_E_ARG;
    }
    if (!guess_kind_matches(c, w->n.kind)) {
      c.last_error = "the network's kind does not match the problem (scalar: Eq. 1 on P1 triangles; "
                     "displacement: Eq. 2 on Q1 quadrilaterals)";
      return NLS_E_ARG;
    }
    GuessCtx* G = new GuessCtx();
    G->net = &w->n;
    G->mode = mode;
    if (w->n.kind == NLS_GUESS_KIND_DISPLACEMENT) G->sweeps = 2;
    build_geometry(c, *G);
    c.dev->guess = G;
  } catch (const std::exception& ex) {
    c.last_error = ex.what();
    guess_free(c);
    return NLS_E_UNSUPPORTED;
  }
  return NLS_OK;
}

int guess_counts(Context& c, int64_t* proposed, int64_t* accepted) {
  GuessCtx* G = c.dev ? (GuessCtx*)c.dev->guess : nullptr;
  if (proposed) *proposed = G ? G->proposed_total : 0;
  if (accepted) *accepted = G ? G->accepted_total : 0;
  if (G) G->proposed_total = G->accepted_total = 0;
  return NLS_OK;
}

}  // namespace nls
