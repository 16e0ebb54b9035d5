// Internal host-side structures of the nls library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "nls.h"

namespace nls {

// Per-subdomain metadata, uploaded verbatim to the device (plain old data).
struct SubMeta {
  int32_t nV;      // table nodes that carry local unknowns (the first nV table nodes)
  int32_t nT;      // all table nodes (nodes touched by the subdomain's elements)
  int32_t n;       // local unknowns = nV * ndof
  int32_t nt;      // table dofs = nT * ndof
  int32_t b;       // half bandwidth of the local matrix over the local unknowns
  int32_t ne;      // elements
  int32_t ncolor;  // element colours (no two elements of one colour share a node)
  int32_t nrows;   // CSR rows: n (local rows only) or nt (full Neumann rows)
  int64_t tnode_off, elem_off, color_off, rowptr_off, nnz_off, nnz, factor_off, vec_off, epos_off;
  int64_t dinv_off;  // packed solve operands of the factors: packed_solve_entries(n, b) entries
};

// Entries of the packed triangular-solve operands of an n x n band factor with half bandwidth b
// (per 32-row block: two 32 x 32 diagonal-block inverses and two 32 x b couplings in FP32; the
// FP64 layout, 16-row blocks, needs at most the same number of entries).
inline int64_t packed_solve_entries(int64_t n, int64_t b) { return ((n + 31) / 32) * (2048 + 64 * b); }

// A batch of subdomain-local problems: overlapping subdomains (rows = local unknowns) or
// non-overlapping ones (rows = all table dofs, for the coarse space).
struct LocalSet {
  int count = 0;
  int ndof = 1, nen = 3;
  bool neumann_rows = false;
  std::vector<SubMeta> meta;
  std::vector<int32_t> tnode_gid;   // table node -> global node
  std::vector<int32_t> elem_gid;    // elements, sorted by (colour, id) per subdomain
  std::vector<int32_t> lconn;       // [elem][nen] table node index
  std::vector<int32_t> color_ptr;   // [ncolor + 1] per subdomain, relative element index
  std::vector<int32_t> rowptr;      // [nrows + 1] per subdomain, relative
  std::vector<int32_t> colidx;      // table dof index
  std::vector<int32_t> epos;        // [elem][(nen*ndof)^2] CSR position (relative), -1 = row not stored
  std::vector<uint8_t> owned;       // per local unknown
  std::vector<int32_t> overlap_sorted_elems;  // elements ascending (for inspection)
  std::vector<int64_t> overlap_sorted_off;
  int64_t total_n = 0, total_nt = 0, total_nnz = 0, total_factor = 0, total_epos = 0, total_dinv = 0;
  int max_n = 0, max_nt = 0, max_b = 0, max_ne = 0, max_nrows = 0;
};

struct DeviceLocalSet {
  int count = 0;
  SubMeta* meta = nullptr;
  int32_t *tnode_gid = nullptr, *elem_gid = nullptr, *lconn = nullptr, *color_ptr = nullptr;
  int32_t *rowptr = nullptr, *colidx = nullptr, *epos = nullptr;
  uint8_t* owned = nullptr;
  double* csr_val = nullptr;       // FP64 local Jacobian (rows per meta.nrows)
  void* factor = nullptr;          // band factors, float or double per precision
  void* dinv = nullptr;            // packed triangular-solve operands of the factors
  double* w = nullptr;             // local states, concatenated (total_n)
  double* work = nullptr;          // three FP64 work vectors per subdomain (3 x total_n)
  int32_t *its = nullptr, *status = nullptr, *chord = nullptr;
  int32_t* order = nullptr;        // processing order (longest first)
  int32_t* queue = nullptr;        // persistent work counter
};

struct Coarse {
  int n_nodes = 0;                 // coarse nodes
  int N0 = 0;                      // coarse dofs
  int b0 = 0;                      // half bandwidth of A_0
  std::vector<int32_t> first_node; // smallest global node id per coarse node
  // P_0 as CSR over global dofs (values filled on the device)
  std::vector<int32_t> p0_rowptr, p0_col;
  std::vector<int64_t> p0_src;     // index into the concatenated Phi blocks
  std::vector<int32_t> p0t_rowptr, p0t_col;  // transpose: rows = coarse dofs, col = global dof
  std::vector<int32_t> p0t_src;    // index into p0 values
  // per non-overlapping subdomain j: columns C_j and dense Phi_j [nt_j x nc_j] (row-major)
  std::vector<int32_t> cj_ptr, cj_col;
  std::vector<int64_t> phi_off;    // offset of Phi_j in the concatenated array
  std::vector<double> phi_host;    // Gamma rows filled on the host, interior rows zero
  int64_t phi_total = 0;
  int max_nc = 0;
  // A_0 (band, FP64) assembly: for band entry e = row * (2 b0 + 1) + (col - row + b0)
  std::vector<int32_t> a0_ptr;     // [N0 * (2b0+1) + 1]
  std::vector<int64_t> a0_src;     // index into concatenated per-subdomain blocks (nc_j^2 each)
  std::vector<int64_t> blk_off;    // offset of subdomain j's nc_j x nc_j block
  int64_t blk_total = 0;
};

struct Context {
  int device = 0;
  void* stream = nullptr;  // cudaStream_t
  bool own_stream = false;
  std::string last_error;
  nls_options opt;
  // problem
  int elem_type = 0, nen = 0, law = 0, ndof = 1;
  int64_t n_nodes = 0, n_elems = 0, N = 0;
  std::vector<double> xy;
  std::vector<int32_t> conn;
  std::vector<uint8_t> dirichlet_node;
  std::vector<int64_t> pending_dirichlet_dofs;
  std::vector<double> pending_dirichlet_vals;
  std::vector<double> ubc;          // Dirichlet values per dof
  std::vector<int32_t> tr_edges;
  std::vector<double> tr_vals;
  double young = 210.0, poisson = 0.3;
  int lambda_mode = NLS_LAMBDA_PRINTED;
  std::vector<double> k_elem, f_elem;
  std::vector<double> f_vol;        // Neo-Hooke volume force per element (fx, fy), load factor 1
  int32_t n_sub = 0, overlap = 1;
  std::vector<int32_t> elem_to_sub;
  int coarse_kind = NLS_COARSE_NONE;
  bool have_mesh = false, have_material = false, have_partition = false, is_setup = false, host_ready = false;
  // setup products (host)
  std::vector<int32_t> owner;
  std::vector<int64_t> star_ptr;
  std::vector<int32_t> star_el;
  LocalSet ov;      // overlapping subdomains
  LocalSet nov;     // non-overlapping subdomains (coarse space)
  Coarse cs;
  std::vector<int32_t> g_color_ptr, g_elem;  // global element colouring
  std::vector<int32_t> g_rowptr, g_col;      // global CSR pattern
  std::vector<int32_t> g_epos;               // [elem][(nen*ndof)^2], element order = conn order
  std::vector<double> geom;                  // per element geometry
  int geom_stride = 0;
  std::vector<double> fext;                  // per dof, load factor 1
  std::vector<uint8_t> free_dof;
  // device memory
  struct Dev* dev = nullptr;
  int64_t device_bytes = 0;
};

// setup.cpp
int build_setup(Context& c);
// Lame parameters of Eq. 2: mu = E / (2 (1 + nu)); lambda as printed, E nu / ((1 + nu)(1 - 2 nu)),
// or its plane-stress reduction 2 mu lambda / (lambda + 2 mu) (NLS_LAMBDA_PLANE_STRESS).
inline void lame(const Context& c, double& mu, double& lam) {
  const double E = c.young, nu = c.poisson;
  mu = E / (2.0 * (1.0 + nu));
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  if (c.lambda_mode == NLS_LAMBDA_PLANE_STRESS) lam = 2.0 * mu * lam / (lam + 2.0 * mu);
}

void build_fext(Context& c);
int device_set_coefficients(Context& c);  // after nls_setup: new k / f on the device, coarse basis rebuilt
int device_upload_fext(Context& c);       // after nls_setup: the rebuilt external load vector to the device
void guess_coefficients_changed(Context& c);
void build_local_set(Context& c, LocalSet& s, int layers, bool neumann_rows, bool keep_overlap_lists);
// solver.cu
int device_setup(Context& c);
void device_free(Context& c);
int solve(Context& c, double* u, int u_dev, nls_report* rep);
int eval_F(Context& c, const double* u, double* F, int is_dev, double load);
int eval_Fx(Context& c, const double* u, double* Fx, int is_dev, double load, int32_t* its, int32_t* st);
int apply_tangent(Context& c, const double* v, double* y, int is_dev);
int get_local_states(Context& c, double* w, int is_dev);
int get_coarse_basis(const Context& c, double* P0);
int get_coarse_matrix(const Context& c, double* A0);
int band_solve(int device, int32_t n, int32_t b, const double* band, const double* rhs, double* x, int32_t precision,
               int32_t method, double* factors_out);
int kernel_stats(const Context& c, int32_t cap, nls_kernel_stat* out, int32_t* n_out);
void reset_kernel_stats(Context& c);
int get_tuning(const Context& c, nls_tuning* out);
void options_changed(Context& c);  // drops state that depends on the options (reused coarse factors, graphs)
int local_corrections_noalloc(Context& c, const double* x, double* Fx, int32_t* its, int32_t* status, double load);
// guess.cu
int guess_attach(Context& c, nls_guess_net* net, int32_t mode);
int guess_counts(Context& c, int64_t* proposed, int64_t* accepted);
// Proposed local starts of one batched local Newton launch (x null: no proposal).
struct GuessProposal {
  const double* x = nullptr;     // concatenated local states
  int32_t* accepted = nullptr;   // per subdomain: 1 if the start was taken
  const double* diag = nullptr;  // per local unknown: sum_e k_e |grad phi_a|^2 |e|
  int sweeps = 0;
  double omega = 0.8;
};
GuessProposal guess_propose(Context& c, const double* x, double load);
GuessProposal guess_smoothing(Context& c);
int guess_features(Context& c, const double* x, double load, float* out);
int guess_decode(Context& c, const double* x, double load, const float* Y, double* out);
int guess_smooth(Context& c, const double* x, double load, const double* w, double* out);
int guess_set_smoothing(Context& c, int32_t sweeps, double omega);
void guess_after_local(Context& c, const double* x, double load, bool proposed);
void guess_free(Context& c);

}  // namespace nls
