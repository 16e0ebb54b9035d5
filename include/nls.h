/*
 * nls.h -- C ABI of the GB300 (sm_103a) two-level nonlinear Schwarz solver.
 *
 * The library solves the discrete nonlinear problem F(u) = 0 of Eq. 3 of Heinlein, Ho,
 * Klawonn, Lanser, "Nonlinear Two-Level Schwarz Methods: A Parallel Implementation in
 * FROSch" (arXiv 2410.24138), for the two model problems of Section 1:
 *   - Eq. 1, nonlinear diffusion -div(k (1 + u^2) grad u) = f on P1 triangles, and
 *   - Eq. 2, compressible Neo-Hooke elasticity on Q1 quadrilaterals (2 dofs per node),
 * by Newton's method on the nonlinearly preconditioned problem F_x(u) = 0 of Section 2:
 * x = one-level (Eq. 5), additive (Eq. 10) or hybrid (Eq. 11), with the local corrections
 * of Eq. 4 on element-overlapping subdomains, the restricted extension of Eq. 8, the RGDSW
 * coarse correction of Eq. 9 and the exact tangents of Eqs. 6 and 12 inside GMRES (Eq. 13).
 *
 * Conventions for every call:
 *   - Every function returns an int status: NLS_OK (0), a negative NLS_E_* error, or a
 *     positive NLS_W_* warning.  nls_strerror() gives a static message; nls_last_error()
 *     gives the detail of the last error on a context.
 *   - The caller owns every array it passes; the library copies what it needs before the
 *     call returns.  Arrays are host pointers unless an argument says "device": then they
 *     must be device memory of the context's device (for example a torch CUDA tensor).
 *   - Global dof numbering: dof = node * ndof + component (ndof = 1 for Eq. 1, 2 for Eq. 2).
 *     Global vectors have n_nodes * ndof entries; entries of Dirichlet dofs hold the
 *     Dirichlet values.
 *   - One context per CUDA stream; calls on a context are not thread safe.
 *   - The library allocates its device memory in nls_setup() and frees it in nls_destroy().
 */
#ifndef NLS_H
#define NLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------- */
#define NLS_OK 0
#define NLS_E_ARG (-1)            /* invalid argument, size or call order */
#define NLS_E_CUDA (-2)           /* a CUDA runtime call failed */
#define NLS_E_NOMEM (-3)          /* device or host allocation failed */
#define NLS_E_UNSUPPORTED (-4)    /* a feature outside the library's scope was requested */
#define NLS_E_LOCAL_NEWTON (-5)   /* a local (Eq. 4) or coarse (Eq. 9) Newton solve failed */
#define NLS_E_PIVOT (-6)          /* zero or non-finite pivot in a no-pivoting band factorization */
#define NLS_E_GMRES (-7)          /* GMRES reached its iteration limit */
#define NLS_E_DIVERGED (-8)       /* non-finite outer residual */
#define NLS_E_DEVICE_TIMEOUT (-9) /* a bounded device-side wait gave up */
#define NLS_W_NOT_CONVERGED 1     /* outer Newton stopped at its iteration limit, or every correction vanished
                                     because local or coarse solves failed */

/* ---- enumerations --------------------------------------------------------------------- */
#define NLS_P1_TRI 1              /* 3-node triangles, nodes counter-clockwise */
#define NLS_Q1_QUAD 2             /* 4-node quadrilaterals, nodes counter-clockwise */
#define NLS_LAW_DIFFUSION 1       /* Eq. 1 */
#define NLS_LAW_NEOHOOKE 2        /* Eq. 2 */
#define NLS_COUPLING_ONE 0        /* F_1 = sum P~_i T_i (Eq. 5, RASPEN form) */
#define NLS_COUPLING_ADD 1        /* F_a (Eq. 10) */
#define NLS_COUPLING_HYBRID 2     /* F_h (Eq. 11) */
#define NLS_COARSE_NONE 0
#define NLS_COARSE_RGDSW 1        /* RGDSW option 2.2 with the Dirichlet-edge modification (Section 2) */
#define NLS_PREC_FP64 0           /* local factorizations and triangular solves in FP64 */
#define NLS_PREC_FP32_IR 1        /* FP32 factorizations + FP64 iterative refinement */

/* Solver options.  nls_options_default() fills the values of Section 3 of the paper:
 * inner Newton rel 1e-5 / abs 1e-11, GMRES rel 1e-6 with at most 1000 iterations. */
typedef struct nls_options {
  int32_t coupling;           /* NLS_COUPLING_* */
  int32_t local_precision;    /* NLS_PREC_* for the local factorizations */
  int32_t coarse_precision;   /* NLS_PREC_* for the coarse factorization */
  int32_t load_steps;         /* dead load ramped as k / load_steps, k = 1..load_steps */
  double outer_atol;          /* outer Newton stops when ||F(u)||_2 < outer_atol */
  int32_t outer_maxit;
  double inner_rtol, inner_atol;   /* local and coarse Newton stopping test */
  int32_t inner_maxit;
  int32_t ls_trials;          /* Armijo backtracking trial steps (alpha = 1, 1/2, ...) */
  double armijo;              /* sufficient decrease constant */
  double gmres_rtol;
  int32_t gmres_restart;
  int32_t gmres_maxit;
  double ir_rtol;             /* iterative refinement stops at ||r - J s|| <= ir_rtol ||r|| */
  int32_t ir_max_sweeps;
  int32_t threads_per_block;  /* CTA size of the batched local Newton kernel, a multiple of 32 in
                                 [64, 256] and at least 32 + the largest half bandwidth (raised to
                                 that if smaller); 0 = library choice (or the autotuner's) */
  int32_t verbose;
  int32_t profile_kernels;    /* 1: time every kernel launch of nls_solve, nls_eval_Fx and
                                 nls_apply_tangent with CUDA events on the context's stream and
                                 accumulate per-kernel totals (nls_get_kernel_stats) */
  int32_t cuda_graphs;        /* 1 (default): a GMRES cycle (up to gmres_restart iterations, each a
                                 tangent application, two Gram-Schmidt passes, the norm and a Givens
                                 step on the device) is one CUDA graph of conditional nodes,
                                 captured once and replayed; the Givens step stops the cycle on the
                                 device, so the host reads its state once per cycle.  0: plain
                                 stream launches and a host check after every iteration.  Graphs are
                                 not used while profile_kernels is set.  Results are identical
                                 either way. */
  int32_t coarse_reuse;       /* 1 (default): the coarse Newton iteration of Eq. 9 starts every
                                 outer step after the first of an nls_solve with the
                                 factorization (and explicit inverse) of the previous tangent
                                 phase's A_0 -- chord steps -- and forms A_0 at
                                 the current point only when a step contracts ||P_0^T F|| by less
                                 than half or fails the line search; 0: a fresh A_0 every coarse
                                 step.  The stopping test (inner_rtol, inner_atol) is the same. */
  int32_t local_reuse;        /* 1 (default): inside nls_solve, from the second F_x evaluation
                                 on, a subdomain whose previous local solve succeeded starts
                                 with chord steps -- Newton steps with the factors (and local
                                 Jacobian) of its previous converged state, which the tangent
                                 kept -- until a step contracts the local residual by less than
                                 a factor 10 or fails the line search; then the Jacobian is
                                 formed at the current state.  The stopping test is the same;
                                 nls_eval_Fx never reuses.  0: a fresh Jacobian every step. */
  int32_t autotune;           /* 1: on the first use, time the batched local Newton kernel with
                                 128- and 256-thread CTAs, the tangent kernel with CTA sizes
                                 from 32 + b to 256 and the coarse band factorization with 256,
                                 512 and 1024 threads on the context's own data, and keep the
                                 fastest (nls_get_tuning).  The choice changes the order of
                                 floating-point reductions only.  0 (default): the library's
                                 fixed choice or threads_per_block. */
  int32_t l2_prefetch;        /* the triangular solves with the packed factors (local Newton
                                 steps, tangent applications, coarse solves) prefetch the
                                 operands of the 32-row block this many blocks ahead into L2;
                                 0 = off, at most 64 (default 4).  Changes no result. */
  int32_t outer_backtrack;    /* 1: the outer Newton step u <- u - alpha du takes the first of
                                 alpha = 1, 1/2, ... (at most min(ls_trials, 5)) with ||F(u')|| <
                                 outer_atol or ||F_x(u')|| <= (1 - armijo alpha) ||F_x(u)||, the last
                                 trial otherwise; an accepted trial's F_x serves the next outer
                                 iteration.  0 (default): always the full step, as in the paper. */
  int32_t coarse_rebuild;     /* 1: inside nls_solve the RGDSW basis is rebuilt at every outer iterate
                                 u from DF(u) (the energy-minimising extension of the same interface
                                 values); 0 (default): built once at setup from DF(u^(0)). */
  int32_t coarse_factor;      /* factorization of the coarse matrix A_0 (Eq. 9), fixed at nls_setup:
                                 NLS_COARSE_FACTOR_AUTO (default): the one-CTA band LU when the half
                                 bandwidth of A_0 is at most 128, the tiled one beyond;
                                 NLS_COARSE_FACTOR_BAND: the band LU in one CTA (half bandwidth of
                                 A_0 at most 128); NLS_COARSE_FACTOR_TILES: a band LU without pivoting
                                 cut into square tiles and spread over many CTAs, with the trailing
                                 tile products of the FP32 form on the tensor cores (TF32 split into
                                 high and low parts, FP32 accumulation) -- for half bandwidths up to
                                 480.  Every coarse solve is refined in FP64 against A_0 either way. */
} nls_options;

#define NLS_COARSE_FACTOR_AUTO 0
#define NLS_COARSE_FACTOR_BAND 1
#define NLS_COARSE_FACTOR_TILES 2

/* Per-solve report. */
typedef struct nls_report {
  int32_t status;                 /* same as the return value of nls_solve */
  int32_t outer_iterations;       /* summed over load steps */
  int32_t gmres_iterations;       /* summed */
  int64_t subdomain_newton_steps; /* sum over outer iterations and subdomains of local Newton iterations */
  int32_t coarse_newton_steps;    /* summed */
  int32_t local_failures;         /* (subdomain, outer iteration) pairs whose local Newton did not converge */
  int32_t first_failed_subdomain; /* -1 if none */
  double final_residual;          /* ||F(u)||_2 at exit */
  double time_total_s;            /* device wall time of nls_solve (CUDA events) */
  double time_inner_s;            /* batched local Newton launches ("Inner solve") */
  double time_coarse_s;           /* coarse Newton and coarse factorizations ("Coarse solve") */
  double time_gmres_s;            /* GMRES incl. tangent applications ("GMRES") */
  double time_other_s;            /* the rest ("Other") */
  int64_t kernel_launches;        /* kernels launched by this call */
  int64_t local_chord_steps;      /* of subdomain_newton_steps, those taken with stored factors
                                     (no Jacobian assembly or factorization; local_reuse) */
} nls_report;

typedef struct nls_ctx nls_ctx;

/* Fill *opt with the defaults described above. */
void nls_options_default(nls_options* opt);

/* Create a context on CUDA device `device`.  Every kernel and copy of the context is issued
 * on `cuda_stream` (a cudaStream_t; NULL selects the legacy default stream).  Device arrays
 * passed to the context must be ready on that stream.  *out receives the context. */
int nls_create(nls_ctx** out, int device, void* cuda_stream);
void nls_destroy(nls_ctx* ctx);
const char* nls_strerror(int status);
const char* nls_last_error(const nls_ctx* ctx);

/* Mesh (Section 1, P1 or Q1): xy [n_nodes * 2] coordinates, conn [n_elems * nen] node ids
 * (nen = 3 for NLS_P1_TRI, 4 for NLS_Q1_QUAD), counter-clockwise. */
int nls_set_mesh(nls_ctx* ctx, int elem_type, int64_t n_nodes, const double* xy, int64_t n_elems,
                 const int32_t* conn);

/* Dirichlet data u = g_D on the listed dofs (Eqs. 1, 2).  All components of a node must be
 * fixed together (NLS_E_UNSUPPORTED otherwise). */
int nls_set_dirichlet(nls_ctx* ctx, int64_t n, const int64_t* dofs, const double* values);

/* Dead-load traction g_N of Eq. 2 on boundary segments: edge_nodes [n_edges * 2],
 * traction [n_edges * 2] force per unit length at load factor 1. */
int nls_set_traction(nls_ctx* ctx, int64_t n_edges, const int32_t* edge_nodes, const double* traction);

/* Dead-load volume force f_vol of Eq. 2 (NLS_LAW_NEOHOOKE; call after nls_set_material):
 * f_vol [n_elems * 2], force per unit area, constant on each element, at load factor 1 (ramped
 * with the traction by the load steps); NULL removes it.  Assembled into the external load
 * vector as int_e f_vol . N_a (2 x 2 Gauss, exact for a constant force on a bilinear element).
 * May follow nls_setup: the load vector is then rebuilt on the device.  NLS_E_ARG for another
 * law or non-finite values. */
int nls_set_volume_force(nls_ctx* ctx, const double* f_vol);

/* Material law.  NLS_LAW_DIFFUSION: params unused, k_elem and f_elem [n_elems] (NULL = 1).
 * NLS_LAW_NEOHOOKE: params = {E, nu}; k_elem, f_elem must be NULL. */
int nls_set_material(nls_ctx* ctx, int law, const double* params, const double* k_elem, const double* f_elem);

/* Which Lame lambda the 2D Neo-Hooke law of Eq. 2 uses with mu = E / (2 (1 + nu)).
 * NLS_LAMBDA_PRINTED (the default, and what nls_set_material restores): the lambda the paper
 * prints, E nu / ((1 + nu)(1 - 2 nu)).  NLS_LAMBDA_PLANE_STRESS: the plane-stress reduction
 * lambda* = 2 mu lambda / (lambda + 2 mu) (= E nu / (1 - nu^2)), for Section 1's "plane stress"
 * taken literally.  Call after nls_set_material and before nls_setup (a later call marks the
 * context as not set up).  NLS_E_ARG for another law or an unknown mode. */
#define NLS_LAMBDA_PRINTED 0
#define NLS_LAMBDA_PLANE_STRESS 1
int nls_set_lambda_mode(nls_ctx* ctx, int mode);

/* Non-overlapping element partition elem_to_sub [n_elems] with ids 0..n_sub-1, grown by
 * `overlap` >= 1 layers of node-sharing elements (Section 2: element-based overlap). */
int nls_set_partition(nls_ctx* ctx, int32_t n_sub, const int32_t* elem_to_sub, int32_t overlap);

/* New per-element coefficients k and f of Eq. 1 (NULL = 1) for a diffusion problem, before or
 * after nls_setup.  After setup only what depends on them is redone -- the external load, the
 * energy-minimising extension of the coarse basis (it uses K = DF(u^(0))) and the learned
 * guess's Jacobi diagonal -- not the index maps, so many coefficient fields can be solved on one
 * mesh and partition (training the learned guess, parameter sweeps).  NLS_E_ARG on a
 * non-finite value or a non-positive k. */
int nls_set_coefficients(nls_ctx* ctx, const double* k_elem, const double* f_elem);

/* Coarse space NLS_COARSE_NONE or NLS_COARSE_RGDSW. */
int nls_set_coarse(nls_ctx* ctx, int kind);

/* Copy the options (validated; NLS_E_ARG on a bad value).  After nls_setup the factor
 * precisions can no longer change (the factor storage is sized for them); any other change
 * takes effect at the next call and drops the reused coarse factorization and the captured
 * GMRES graphs. */
int nls_set_options(nls_ctx* ctx, const nls_options* opt);
int nls_get_options(const nls_ctx* ctx, nls_options* opt);

/* Build every map (overlap, local numbering, owners, coarse interface classes), upload to the
 * device and compute the coarse basis.  Must follow the nls_set_* calls above. */
int nls_setup(nls_ctx* ctx);

/* Host part of nls_setup only: builds every integer map (overlap, local numbering, owners,
 * coarse interface classes) without touching a GPU.  The inspection calls nls_get_sizes,
 * nls_get_local_dofs, nls_get_overlap_elems, nls_get_owners and nls_get_coarse_nodes work
 * after it; nls_solve and the evaluation hooks need nls_setup. */
int nls_setup_host(nls_ctx* ctx);

/* Solve F(u) = 0 by the outer Newton iteration on F_x (Eq. 13).  u_inout [n_nodes * ndof]:
 * initial guess in, solution out (Dirichlet entries are overwritten with the Dirichlet values);
 * host memory, or device memory when u_is_device != 0.  rep may be NULL. */
int nls_solve(nls_ctx* ctx, double* u_inout, int u_is_device, nls_report* rep);

/* ---- parity and inspection hooks ------------------------------------------------------- */

/* Sizes of the setup products. */
typedef struct nls_sizes {
  int64_t n_nodes, n_dofs, n_elems;
  int32_t ndof, n_sub, n_coarse_nodes, n_coarse_dofs;
  int64_t total_local_dofs;   /* sum_i |V_i| */
  int64_t total_overlap_elems;
  int32_t max_local_dofs, max_half_band, coarse_half_band;
  int64_t device_bytes;
  int64_t total_factor_entries;  /* sum_i |V_i| (2 b_i + 1): band factor storage of all subdomains */
  int64_t total_local_nnz;       /* sum_i nnz(R_i DF P_i plus its boundary columns) */
  int64_t total_table_dofs;      /* sum_i dofs touched by Omega_i' */
  int32_t factor_bytes;          /* 4 (FP32 factors) or 8 (FP64 factors) per the current options */
  int32_t pad;
  int64_t total_solve_entries;   /* sum_i entries of the packed triangular-solve operands that one
                                    pair of triangular solves reads (diagonal-block inverses and
                                    couplings, blocks of 32 rows in FP32 and 16 rows in FP64) */
  double lu_flops;               /* sum_i flops of one no-pivoting band LU of subdomain i:
                                    sum_k (lim_k + 2 lim_k^2), lim_k = min(b_i, n_i - 1 - k) */
  double solve_flops;            /* sum_i flops of one forward + backward solve with the packed
                                    operands: 2 entries read = 2 flops per entry used */
} nls_sizes;

/* Per-kernel timing collected while nls_options.profile_kernels is set.  `name` is a static
 * string owned by the library. */
typedef struct nls_kernel_stat {
  const char* name;
  int64_t launches;
  double total_ms;
} nls_kernel_stat;
/* Copy up to `cap` entries (kernels with at least one launch) into out; *n_out receives the count. */
int nls_get_kernel_stats(const nls_ctx* ctx, int32_t cap, nls_kernel_stat* out, int32_t* n_out);

/* CTA sizes in use for the batched local Newton kernel, the tangent kernel and the coarse
 * factorization, and whether they came from the autotuner (1) or the fixed rule (0).  Valid
 * after nls_setup. */
typedef struct nls_tuning {
  int32_t newton_threads, apply_threads;
  int32_t newton_tuned, apply_tuned;
  double newton_ms[2];        /* measured launch times of the 128- and 256-thread variants (0: not tried) */
  int32_t graphs_captured;    /* GMRES cycle graphs currently instantiated (0 or 1) */
  int32_t coarse_threads;     /* CTA size of the coarse band factorization (autotuned when enabled) */
} nls_tuning;
int nls_get_tuning(const nls_ctx* ctx, nls_tuning* out);
int nls_reset_kernel_stats(nls_ctx* ctx);
int nls_get_sizes(const nls_ctx* ctx, nls_sizes* out);

/* Local numbering of subdomain `sub` (R_i of Section 2): the global dof ids of its local
 * unknowns in local order (ascending), dofs_out[cap]; owned_out[cap] (may be NULL) receives 1
 * where P~_i keeps the dof (Eq. 8).  *n_out receives |V_i|. */
int nls_get_local_dofs(const nls_ctx* ctx, int32_t sub, int64_t cap, int64_t* dofs_out, uint8_t* owned_out,
                       int64_t* n_out);
/* Elements of the overlapping subdomain Omega_i' (ascending global ids). */
int nls_get_overlap_elems(const nls_ctx* ctx, int32_t sub, int64_t cap, int32_t* elems_out, int64_t* n_out);
/* owner(node) of every node (min id of the non-overlapping subdomains touching it). */
int nls_get_owners(const nls_ctx* ctx, int32_t* owners_out);
/* Coarse nodes: for coarse node c, its smallest global node id (ascending order). */
int nls_get_coarse_nodes(const nls_ctx* ctx, int32_t* first_node_out);
/* The coarse basis P_0 as a dense column-major [n_dofs x n_coarse_dofs] host array. */
int nls_get_coarse_basis(const nls_ctx* ctx, double* P0_out);

/* The coarse matrix A_0 = P_0^T DF(u_0) P_0 of Eq. 9 formed by the last tangent phase (or coarse
 * Newton step) in FP64 band storage: A0_out [n_coarse_dofs x (2 coarse_half_band + 1)], entry
 * (i, i - b0 + d) at i (2 b0 + 1) + d. */
int nls_get_coarse_matrix(const nls_ctx* ctx, double* A0_out);

/* The coarse factorization and solve of Eq. 9 applied to a given band matrix (parity hook and
 * utility).  band [n x (2b + 1)] (host, FP64, entry (i, i - b + d) at i (2b + 1) + d; entries
 * outside the matrix are ignored) is factored without pivoting by `method`
 * (NLS_COARSE_FACTOR_BAND, _TILES, or _AUTO as in nls_options.coarse_factor) in `precision`
 * (NLS_PREC_FP64, or NLS_PREC_FP32_IR: FP32 factors, each solve refined in FP64 against the band
 * until ||rhs - A x|| <= 1e-10 ||rhs||, at most 5 sweeps), then A x = rhs is solved; x [n] and
 * rhs [n] are host arrays.  factors_out [n x (2b + 1)] (may be NULL) receives the factors in the
 * band layout: d < b the multipliers of the unit lower factor L, d = b the reciprocal pivots
 * 1 / U_ii, d > b the entries of U.  Runs on `device`'s legacy default stream with its own
 * memory, freed before returning.  NLS_E_PIVOT for a zero or non-finite pivot,
 * NLS_E_UNSUPPORTED beyond the half bandwidths the methods take (BAND 128, and a window of
 * (b + 10) rows that fits in shared memory: about 160 in FP32, 110 in FP64; TILES 480) or when
 * the solve vector (n values) does not fit in shared memory. */
int nls_band_solve(int device, int32_t n, int32_t b, const double* band, const double* rhs, double* x,
                   int32_t precision, int32_t method, double* factors_out);

/* F(u) of Eq. 3 (Dirichlet rows zero) at load factor `load`; u, F of length n_dofs. */
int nls_eval_F(nls_ctx* ctx, const double* u, double* F, int is_device, double load);

/* F_x(u) (Eq. 5, 10 or 11 per the coupling option) at load factor `load`, and keep the
 * linearisation for nls_apply_tangent.  local_its_out [n_sub] and local_status_out [n_sub]
 * (may be NULL) receive the local Newton iteration counts and status (0 = converged,
 * 1 = iteration limit, 2 = line search failed, 3 = non-finite, 4 = bad pivot). */
int nls_eval_Fx(nls_ctx* ctx, const double* u, double* Fx, int is_device, double load,
                int32_t* local_its_out, int32_t* local_status_out);

/* y = DF_x(u) v (Eqs. 6, 12) at the u of the last nls_eval_Fx. */
int nls_apply_tangent(nls_ctx* ctx, const double* v, double* y, int is_device);

/* Converged local states w_i = R_i (u - P_i T_i(u)) of the last nls_eval_Fx, concatenated in
 * subdomain order (total_local_dofs entries). */
int nls_get_local_states(nls_ctx* ctx, double* w_out, int is_device);

/* ---- learned initial guess (not in the paper) ------------------------------------------
 * A small fully connected network proposes the starting point of every local Newton solve
 * (Eq. 4), on structured meshes of the unit square (n x n cells, nodes numbered row by row).
 * Box of a subdomain: the grid rectangle one node beyond its local unknowns, clamped to the mesh
 * (for Eq. 1 the ring of Dirichlet data around the unknowns; a side on a Neumann edge of Eq. 2 is
 * that edge).  Two kinds of network:
 * - scalar (Eq. 1, P1 triangles): 391 inputs per subdomain -- x on the four sides of the box,
 *   sampled at 33 points each, log k on 16 x 16 points of the box, the load factor times f, and
 *   the box width and height; 1024 outputs.
 * - displacement (Eq. 2, Q1 quadrilaterals): 267 inputs -- the 4 x 33 side samples of the first
 *   and of the second displacement component, the load factor, the box width and height; 2048
 *   outputs (1024 per component).
 * Each 1024 outputs are a 32 x 32 correction, on a canonical grid of the box, to the Coons
 * (bilinear transfinite) patch of one component's side data; the guess at a node is the patch
 * plus the bilinearly interpolated correction.  Layers: n_in -> h1 -> h2 -> n_out, tanh-form
 * GELU.  Training: BF16 operands on the tensor cores with FP32 accumulation, FP32 master
 * weights, Adam, loss 1/(2B) sum ||y - t||^2 on normalised inputs and targets.  Inference: FP32.
 * Before the test, `sweeps` damped Jacobi steps w <- w - omega r(w) / d(w) on the local
 * problem remove the pointwise (high-frequency) part of the network's error, which otherwise
 * dominates the residual.  Eq. 1: d_a(w) = (1 + w_a^2) sum_{e owns a} k_e |grad phi_a|^2 |e|,
 * the diagonal of the Jacobian's leading term; Eq. 2: d the diagonal of the linear-elastic
 * stiffness (the tangent at zero displacement).  Defaults: omega = 0.8 (the damping that
 * minimises the smoothing factor of Jacobi on the five-point stencil P1 yields here) and 6 sweeps
 * for the scalar kind, 2 for the displacement kind (measured best on held-out partitions of the
 * Neo-Hooke workload: more sweeps cost more local residuals than they save Newton steps).
 * A guess is used only where its (smoothed) local residual is smaller than that of R_i x (the
 * start the method uses otherwise); the local stopping test stays relative to the residual at
 * R_i x, so convergence to tolerance does not depend on the network.
 * The network lives on one device; every array below is a host pointer. */
typedef struct nls_guess_net nls_guess_net;
#define NLS_GUESS_FEATURES 391        /* inputs of the scalar kind */
#define NLS_GUESS_OUTPUTS 1024        /* outputs of the scalar kind */
#define NLS_GUESS_FEATURES_DISP 267   /* inputs of the displacement kind */
#define NLS_GUESS_OUTPUTS_DISP 2048   /* outputs of the displacement kind */
#define NLS_GUESS_KIND_SCALAR 0
#define NLS_GUESS_KIND_DISPLACEMENT 1
#define NLS_GUESS_USE 1      /* propose starting points in nls_solve / nls_eval_Fx */
#define NLS_GUESS_HARVEST 2  /* record (features, converged local state) pairs after every local solve */
#define NLS_GUESS_FIRST_OUTER 4  /* with NLS_GUESS_USE: propose only at the first outer iteration of each
                                    load step of nls_solve (later iterations start from R_i u) */

/* Create a network of NLS_GUESS_KIND_* `kind` with hidden widths h1, h2 (multiples of 16),
 * weights drawn from splitmix64 `seed`, on `device`, with room for `capacity` training pairs.
 * nls_guess_create makes the scalar kind.  NLS_E_ARG on a bad kind, width or capacity. */
int nls_guess_create(nls_guess_net** out, int device, int32_t h1, int32_t h2, uint64_t seed, int64_t capacity);
int nls_guess_create_kind(nls_guess_net** out, int device, int32_t kind, int32_t h1, int32_t h2, uint64_t seed,
                          int64_t capacity);
/* The network's kind and its numbers of inputs and outputs (n_in, n_out below). */
int nls_guess_dims(const nls_guess_net* net, int32_t* kind, int32_t* n_in, int32_t* n_out);
void nls_guess_destroy(nls_guess_net* net);
/* Attach a network to a context (after nls_setup) with NLS_GUESS_* mode bits, or detach (net NULL).
 * NLS_E_ARG when the kind does not match the problem (scalar: Eq. 1 on P1 triangles;
 * displacement: Eq. 2 on Q1 quadrilaterals); NLS_E_UNSUPPORTED when the mesh is not a structured
 * grid of the unit square numbered row by row. */
int nls_guess_attach(nls_ctx* ctx, nls_guess_net* net, int32_t mode);
/* Train on the harvested pairs: `steps` Adam steps on random minibatches of `batch` pairs
 * (splitmix64 `seed`), learning rate lr.  loss_out[steps] (may be NULL) receives the losses. */
int nls_guess_train(nls_guess_net* net, int32_t steps, int32_t batch, double lr, uint64_t seed, float* loss_out);
/* Number of harvested pairs. */
int nls_guess_pairs(const nls_guess_net* net, int64_t* n_out);
/* Parameters as one FP32 array in the order W1 [h1 x n_in], b1, W2 [h2 x h1], b2, W3 [n_out x h2],
 * b3 (row-major); *count receives the length.  set_params also resets the Adam state. */
int nls_guess_get_params(const nls_guess_net* net, float* params, int64_t* count);
int nls_guess_set_params(nls_guess_net* net, const float* params, int64_t count);
/* Normalisation of inputs and targets: x_norm = (x - mean) / scale per input (mean, scale [n_in]),
 * t_norm = t / tscale. */
int nls_guess_get_normalisation(const nls_guess_net* net, float* mean, float* scale, float* tscale);
int nls_guess_set_normalisation(nls_guess_net* net, const float* mean, const float* scale, float tscale);
/* Gradient of the loss on a given batch of normalised inputs X [B x n_in] and targets
 * T [B x n_out] (host arrays), in the parameter order above, with FP32 (precision 0) or BF16
 * (precision 1) GEMM operands; *loss receives the loss.  Test hook for the gradient checks. */
int nls_guess_gradient(nls_guess_net* net, int32_t B, const float* X, const float* T, int32_t precision, float* grad,
                       float* loss);
/* Network output (FP32 inference) for normalised inputs X [B x n_in] into Y [B x n_out]. */
int nls_guess_forward(nls_guess_net* net, int32_t B, const float* X, float* Y);
/* Test hooks of the input and output maps (context with an attached network; x [n_dofs] host):
 * the raw inputs of every subdomain at x and load factor `load` (before normalisation) into
 * features_out [n_sub x n_in] (FP32); the proposal decoded from given network outputs
 * Y [n_sub x n_out] (normalised units, FP32) at x into guess_out [total_local_dofs] (the local
 * unknowns of every subdomain, concatenated in subdomain order as nls_get_local_states); and the
 * smoothing of given starts w [total_local_dofs] at x into w_out [total_local_dofs], with the
 * attached network's smoothing parameters. */
int nls_guess_features(nls_ctx* ctx, const double* x, double load, float* features_out);
int nls_guess_decode(nls_ctx* ctx, const double* x, double load, const float* Y, double* guess_out);
int nls_guess_smooth(nls_ctx* ctx, const double* x, double load, const double* w, double* w_out);
/* Guesses proposed and accepted by the local solves since the last call (then reset). */
int nls_guess_counts(nls_ctx* ctx, int64_t* proposed, int64_t* accepted);
/* Smoothing of proposed starts (see above): sweeps in [0, 64], omega in (0, 1].  Needs an
 * attached network; attaching resets the defaults. */
int nls_guess_set_smoothing(nls_ctx* ctx, int32_t sweeps, double omega);

/* ---- allocation-free variant (the paper has no counterpart) ----------------------------
 * Local corrections F_1(x) = sum_i P~_i T_i(x) of the context's overlapping subdomains -- the
 * same batched local-Newton kernel as nls_eval_Fx with the one-level coupling, without the
 * coarse correction and without keeping a tangent -- computed without allocating anything.
 * It exists for callers that cannot allocate device memory at the time they need the
 * corrections: code being recorded into a CUDA graph (no cudaMalloc during stream capture),
 * applications whose own memory manager owns the GPU, and loops that must not risk the
 * implicit synchronisation of cudaMalloc / cudaFree.  The kernel's scratch (local Jacobians,
 * band factors, packed solve operands, local states, work vectors, work counter) lives in a
 * 32 MiB device array compiled into the
 * library, which every GPU that loads the library keeps until the process exits.
 *   x   [n_dofs] device input (the point, Dirichlet entries holding the Dirichlet values);
 *   Fx  [n_dofs] device output; every entry is written (Dirichlet entries with 0);
 *   its, status [n_sub] optional device outputs (NULL: kept in the scratch area);
 *   load  external-load factor.
 * Requires a context after nls_setup; returns NLS_E_ARG, with the byte counts in
 * nls_last_error, when the problem needs more scratch than the array holds.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents; calls whose work overlaps on the GPU race on it.  Work is issued on the
 * context's stream and the call does not synchronise. */
int nls_local_corrections_noalloc(nls_ctx* ctx, const double* x, double* Fx, int32_t* its, int32_t* status,
                                  double load);

#ifdef __cplusplus
}
#endif
#endif /* NLS_H */
