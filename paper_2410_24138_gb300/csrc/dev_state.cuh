// Device-side state of one solver context and the launch / error helpers shared by the
// translation units that launch kernels (solver.cu, guess.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "nls_internal.h"

namespace nls {

struct CudaFailure : std::runtime_error {
  explicit CudaFailure(const std::string& s) : std::runtime_error(s) {}
};
// A kernel's bounded wait gave up (NLS_E_DEVICE_TIMEOUT); the context stays usable.
struct DeviceTimeout : std::runtime_error {
  explicit DeviceTimeout(const std::string& s) : std::runtime_error(s) {}
};

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) throw ::nls::CudaFailure(std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define LAUNCH(D, kernel, grid, block, smem, ...) LAUNCH_NAMED(D, #kernel, kernel, grid, block, smem, __VA_ARGS__)

// The same with the profiling name given as a static string (for kernels launched through a
// template whose stringified name would show the template parameters' names).
#define LAUNCH_NAMED(D, name, kernel, grid, block, smem, ...)             \
  do {                                                                     \
    const bool prof_ = (D).prof;                                           \
    if (prof_) (D).prof_begin(name);                                       \
    kernel<<<(grid), (block), (smem), (D).s>>>(__VA_ARGS__);               \
    if (prof_) (D).prof_end();                                             \
    (D).launches += 1;                                                     \
    CK(cudaGetLastError());                                                \
  } while (0)

// Status words of the local and coarse solves (per subdomain, and of the coarse factorization).
// ST_TIMEOUT: a bounded device-side wait gave up (the kernel returned without finishing).
enum LocalStatus { ST_OK = 0, ST_MAXIT = 1, ST_LS = 2, ST_NONFINITE = 3, ST_PIVOT = 4, ST_TIMEOUT = 9 };

// State of one GMRES cycle on the device (32 bytes).
struct GmresState {
  int j;          // iterations done in the current cycle
  int done;       // 1: converged (|g_j| <= target), breakdown or a non-finite norm
  int limit;      // iterations allowed in this cycle
  int pad;
  double target;  // the cycle stops once |g_j| <= target
  double res;     // |g_j| after the last iteration (the residual norm of the least-squares problem)
};

// Tiled band LU of the coarse matrix A_0 (coarse_tlu.cu): square tiles of TS x TS, tile row i
// holding tiles j = i - TB .. i + TB (SW = 2 TB + 1 slots; slots outside the matrix unused).
struct TileLU {
  int TS = 0, NT = 0, TB = 0, SW = 0;
  bool f32 = true;
  void* T = nullptr;   // tiles: slot (i, j - i + TB), TS x TS values; j <= i row-major, j > i transposed
  void* DG = nullptr;  // factored diagonal tiles (unit L below the diagonal, U on and above it)
  CUtensorMap map;     // FP32 tiles as a 2D tensor of rows of TS values (TMA, 32 x TS boxes)
  bool solve_tiles = false;  // FP32: inverted diagonal tiles and solve products for the cluster solve
  int32_t* solve_status = nullptr;  // ST_TIMEOUT once a cluster solve gave up waiting (else 0)
  int64_t launches_per_factor = 0;
};

// ------------------------------------------------------------------------------------------
// device state
// ------------------------------------------------------------------------------------------
struct Dev {
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t launches = 0;
  int nsm = 152;
  size_t smem_optin = 0;
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    CK(cudaMalloc(&p, n * sizeof(T)));
    allocs.push_back(p);
    bytes += (int64_t)(n * sizeof(T));
    return (T*)p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return p;
  }
  void release(void* p) {
    for (auto& q : allocs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
  // mesh
  int32_t *conn = nullptr, *g_elem = nullptr, *g_rowptr = nullptr, *g_col = nullptr, *g_epos = nullptr;
  int64_t* star_ptr = nullptr;  // node stars (ascending element ids) for the global residual's node sums
  int32_t* star_ref = nullptr;  // e nen + a per star entry
  double* Re = nullptr;         // element residuals [e][a][dof]
  double *geom = nullptr, *kcoef = nullptr, *fext = nullptr, *ubc = nullptr, *g_val = nullptr;
  uint8_t* free_dof = nullptr;
  DeviceLocalSet ov, nov;
  // coarse
  int32_t *p0_rowptr = nullptr, *p0_col = nullptr, *p0t_rowptr = nullptr, *p0t_col = nullptr, *p0t_src = nullptr;
  int64_t* p0_src = nullptr;
  double *p0_val = nullptr, *p0t_val = nullptr, *phi = nullptr, *Y = nullptr, *blk = nullptr, *A0 = nullptr;
  int64_t *phi_off = nullptr, *blk_off = nullptr, *a0_src = nullptr;
  int32_t *cj_ptr = nullptr, *a0_ptr = nullptr;
  void* A0f = nullptr;
  void* A0dinv = nullptr;
  TileLU* tlu = nullptr;  // tiled coarse factorization (when in use)
  int32_t* cstatus = nullptr;
  // vectors
  double* ut = nullptr;  // trial point of the outer backtracking
  double *u = nullptr, *x = nullptr, *u0 = nullptr, *Fx = nullptr, *F = nullptr, *t1 = nullptr, *t2 = nullptr,
         *w0 = nullptr, *gx = nullptr;
  double *c = nullptr, *ct = nullptr, *dc = nullptr, *g = nullptr, *gt = nullptr, *cres = nullptr, *tg = nullptr;
  void* cy = nullptr;
  double *V = nullptr, *partial = nullptr, *scal = nullptr, *coef = nullptr;
  // GMRES least-squares state on the device: R (m x m), rotations, rotated right-hand side, state
  double *gR = nullptr, *gcs = nullptr, *gsn = nullptr, *gg = nullptr;
  GmresState* gst = nullptr;
  int* bad = nullptr;
  unsigned long long* phase = nullptr;  // k_local_newton phase clocks (profiling)
  void* ainv = nullptr;                 // explicit A_0^-1 (transposed, factor precision) for the tangent phase
  double* gpart = nullptr;              // GEMV chunk partials
  double* cpart = nullptr;              // refinement of the explicit-inverse solves: per-CTA partial norms
  int* cflag = nullptr;                 // [0] refinement converged, [1] ticket counter
  bool ainv_valid = false;
  bool coarse_fact_valid = false;  // the coarse band factors hold A_0 at some earlier point
  bool local_factors_valid = false;  // the local factors hold the previous evaluation's tangent factors
  bool local_reuse_active = false;   // chord steps allowed (inside nls_solve with local_reuse)
  int clock_khz = 1;
  double* h_scal = nullptr;  // pinned
  int m = 0;                 // GMRES restart length allocated
  bool tangent_ready = false;
  void* guess = nullptr;  // learned-guess attachment (guess.cu)
  double last_load = 1.0;
  // CTA sizes (0 = fixed rule) and the autotuner's measurements
  int newton_T = 0, apply_T = 0, coarse_T = 1024;
  bool newton_tuned = false, apply_tuned = false, coarse_tuned = false;
  double newton_ms[2] = {0.0, 0.0};
  // GMRES iteration graphs, one per Krylov index, valid while `graph_key` matches
  cudaStream_t cap = nullptr;  // private stream the graphs are captured on
  cudaStream_t s2 = nullptr;   // second stream: the tangent phase's coarse work
  bool coarse_beside = false;
  int outer_k = 0;  // outer iteration of the current load step inside nls_solve (-1 outside)  // a coarse factorization runs on s2 during the next local Newton launch
  cudaEvent_t ev_u0 = nullptr, ev_coarse = nullptr;
  std::vector<cudaGraphExec_t> it_exec;
  std::vector<int64_t> it_launches;
  std::string graph_key;
  void reset_graphs() {
    for (auto& g : it_exec)
      if (g) cudaGraphExecDestroy(g);
    it_exec.clear();
    it_launches.clear();
    graph_key.clear();
  }
  // per-launch CUDA-event timing (nls_options.profile_kernels)
  bool prof = false;
  struct EvRec {
    cudaEvent_t a, b;
    const char* name;
  };
  std::vector<EvRec> evs;
  size_t ev_used = 0;
  struct Stat {
    std::string name;
    int64_t launches;
    double ms;
  };
  std::vector<Stat> stats;
  void prof_begin(const char* name) {
    if (ev_used == evs.size()) {
      EvRec r;
      CK(cudaEventCreate(&r.a));
      CK(cudaEventCreate(&r.b));
      evs.push_back(r);
    }
    evs[ev_used].name = name;
    CK(cudaEventRecord(evs[ev_used].a, s));
  }
  void prof_end() {
    CK(cudaEventRecord(evs[ev_used].b, s));
    ++ev_used;
    if (ev_used >= 65536) prof_flush();
  }
  void prof_flush() {
    if (!ev_used) return;
    CK(cudaDeviceSynchronize());  // events may sit on the second stream too (profiling mode only)
    for (size_t i = 0; i < ev_used; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, evs[i].a, evs[i].b));
      Stat* st = nullptr;
      for (auto& x : stats)
        if (x.name == evs[i].name) st = &x;
      if (!st) {
        stats.push_back(Stat{evs[i].name, 0, 0.0});
        st = &stats.back();
      }
      st->launches += 1;
      st->ms += ms;
    }
    ev_used = 0;
  }
};

}  // namespace nls
