// C ABI entry points (include/nls.h): argument checking, copies of the caller's arrays, and
// dispatch to the setup (setup.cpp) and the device solver (solver.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>

#include "nls_internal.h"

using nls::Context;

struct nls_ctx {
  Context c;
};

namespace {

int fail(nls_ctx* ctx, int code, const char* msg) {
  if (ctx) ctx->c.last_error = msg;
  return code;
}

}  // namespace

extern "C" {

void nls_options_default(nls_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->coupling = NLS_COUPLING_HYBRID;
  o->local_precision = NLS_PREC_FP32_IR;
  o->coarse_precision = NLS_PREC_FP64;
  o->load_steps = 1;
  o->outer_atol = 1e-8;
  o->outer_maxit = 30;
  o->inner_rtol = 1e-5;
  o->inner_atol = 1e-11;
  o->inner_maxit = 50;
  o->ls_trials = 10;
  o->armijo = 1e-4;
  o->gmres_rtol = 1e-6;
  o->gmres_restart = 50;
  o->gmres_maxit = 1000;
  o->ir_rtol = 1e-10;
  o->ir_max_sweeps = 5;
  o->threads_per_block = 0;
  o->cuda_graphs = 1;
  o->coarse_reuse = 1;
  o->local_reuse = 1;
  o->autotune = 0;
  o->l2_prefetch = 4;
  o->outer_backtrack = 0;
  o->coarse_rebuild = 0;
  o->coarse_factor = NLS_COARSE_FACTOR_AUTO;
  o->verbose = 0;
}

const char* nls_strerror(int s) {
  switch (s) {
    case NLS_OK: return "ok";
    case NLS_E_ARG: return "invalid argument or call order";
    case NLS_E_CUDA: return "CUDA runtime error";
    case NLS_E_NOMEM: return "out of memory";
    case NLS_E_UNSUPPORTED: return "unsupported feature";
    case NLS_E_LOCAL_NEWTON: return "local or coarse Newton solve failed";
    case NLS_E_PIVOT: return "zero or non-finite pivot in a band factorization";
    case NLS_E_GMRES: return "GMRES reached its iteration limit";
    case NLS_E_DIVERGED: return "outer iteration produced a non-finite residual";
    case NLS_E_DEVICE_TIMEOUT: return "bounded device wait gave up";
    case NLS_W_NOT_CONVERGED: return "outer Newton reached its iteration limit";
    default: return "unknown status";
  }
}

const char* nls_last_error(const nls_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : ""; }

int nls_create(nls_ctx** out, int device, void* stream) {
  if (!out) return NLS_E_ARG;
  nls_ctx* ctx = new (std::nothrow) nls_ctx();
  if (!ctx) return NLS_E_NOMEM;
  ctx->c.device = device;
  ctx->c.stream = stream;
  nls_options_default(&ctx->c.opt);
  *out = ctx;
  return NLS_OK;
}

void nls_destroy(nls_ctx* ctx) {
  if (!ctx) return;
  nls::device_free(ctx->c);
  delete ctx;
}

int nls_set_mesh(nls_ctx* ctx, int elem_type, int64_t n_nodes, const double* xy, int64_t n_elems, const int32_t* conn) {
  if (!ctx) return NLS_E_ARG;
  if (elem_type != NLS_P1_TRI && elem_type != NLS_Q1_QUAD) return fail(ctx, NLS_E_ARG, "unknown element type");
  if (n_nodes <= 0 || n_elems <= 0 || !xy || !conn) return fail(ctx, NLS_E_ARG, "empty mesh");
  if (n_nodes > INT32_MAX || n_elems > INT32_MAX) return fail(ctx, NLS_E_UNSUPPORTED, "mesh larger than 2^31 entities");
  Context& c = ctx->c;
  c.elem_type = elem_type;
  c.nen = (elem_type == NLS_P1_TRI) ? 3 : 4;
  c.n_nodes = n_nodes;
  c.n_elems = n_elems;
  c.xy.assign(xy, xy + 2 * n_nodes);
  c.conn.assign(conn, conn + c.nen * n_elems);
  for (int32_t v : c.conn)
    if (v < 0 || v >= n_nodes) return fail(ctx, NLS_E_ARG, "connectivity refers to a node out of range");
  c.dirichlet_node.assign(n_nodes, 0);
  c.have_mesh = true;
  c.is_setup = false;
  return NLS_OK;
}

int nls_set_dirichlet(nls_ctx* ctx, int64_t n, const int64_t* dofs, const double* values) {
  if (!ctx || !ctx->c.have_mesh) return fail(ctx, NLS_E_ARG, "set the mesh first");
  if (n < 0 || (n > 0 && !dofs)) return fail(ctx, NLS_E_ARG, "bad Dirichlet arrays");
  Context& c = ctx->c;
  c.pending_dirichlet_dofs.assign(dofs, dofs + n);
  c.pending_dirichlet_vals.assign(n, 0.0);
  if (values) c.pending_dirichlet_vals.assign(values, values + n);
  c.is_setup = false;
  return NLS_OK;
}

int nls_set_traction(nls_ctx* ctx, int64_t n_edges, const int32_t* edge_nodes, const double* traction) {
  if (!ctx || !ctx->c.have_mesh) return fail(ctx, NLS_E_ARG, "set the mesh first");
  if (n_edges < 0 || (n_edges > 0 && (!edge_nodes || !traction))) return fail(ctx, NLS_E_ARG, "bad traction arrays");
  Context& c = ctx->c;
  c.tr_edges.assign(edge_nodes, edge_nodes + 2 * n_edges);
  c.tr_vals.assign(traction, traction + 2 * n_edges);
  for (int32_t v : c.tr_edges)
    if (v < 0 || v >= c.n_nodes) return fail(ctx, NLS_E_ARG, "traction edge refers to a node out of range");
  c.is_setup = false;
  return NLS_OK;
}

int nls_set_volume_force(nls_ctx* ctx, const double* f_vol) {
  if (!ctx || !ctx->c.have_material) return fail(ctx, NLS_E_ARG, "set the material first");
  Context& c = ctx->c;
  if (c.law != NLS_LAW_NEOHOOKE) return fail(ctx, NLS_E_ARG, "the volume force applies to the Neo-Hooke law");
  if (f_vol)
    for (int64_t k = 0; k < 2 * c.n_elems; ++k)
      if (!std::isfinite(f_vol[k])) return fail(ctx, NLS_E_ARG, "non-finite volume force");
  c.f_vol.clear();
  if (f_vol) c.f_vol.assign(f_vol, f_vol + 2 * c.n_elems);
  if (!c.is_setup) return NLS_OK;
  nls::build_fext(c);
  if (!c.dev) return NLS_OK;  // host-only setup
  const int st = nls::device_upload_fext(c);
  if (st != NLS_OK) return fail(ctx, st, c.last_error.c_str());
  return NLS_OK;
}

int nls_set_material(nls_ctx* ctx, int law, const double* params, const double* k_elem, const double* f_elem) {
  if (!ctx || !ctx->c.have_mesh) return fail(ctx, NLS_E_ARG, "set the mesh first");
  Context& c = ctx->c;
  if (law == NLS_LAW_DIFFUSION) {
    if (c.elem_type != NLS_P1_TRI) return fail(ctx, NLS_E_UNSUPPORTED, "the diffusion law is implemented on P1 triangles");
    c.ndof = 1;
    c.k_elem.clear();
    c.f_elem.clear();
    if (k_elem) c.k_elem.assign(k_elem, k_elem + c.n_elems);
    if (f_elem) c.f_elem.assign(f_elem, f_elem + c.n_elems);
  } else if (law == NLS_LAW_NEOHOOKE) {
    if (c.elem_type != NLS_Q1_QUAD) return fail(ctx, NLS_E_UNSUPPORTED, "the Neo-Hooke law is implemented on Q1 quadrilaterals");
    if (!params) return fail(ctx, NLS_E_ARG, "Neo-Hooke needs params = {E, nu}");
    if (k_elem || f_elem) return fail(ctx, NLS_E_ARG, "k_elem / f_elem apply to the diffusion law only");
    c.ndof = 2;
    c.young = params[0];
    c.poisson = params[1];
    if (!(c.young > 0) || !(c.poisson > -1.0 && c.poisson < 0.5)) return fail(ctx, NLS_E_ARG, "invalid E or nu");
  } else {
    return fail(ctx, NLS_E_ARG, "unknown material law");
  }
  c.law = law;
  c.f_vol.clear();
  c.lambda_mode = NLS_LAMBDA_PRINTED;
  c.have_material = true;
  c.is_setup = false;
  return NLS_OK;
}

int nls_set_lambda_mode(nls_ctx* ctx, int mode) {
  if (!ctx || !ctx->c.have_material) return fail(ctx, NLS_E_ARG, "set the material first");
  Context& c = ctx->c;
  if (c.law != NLS_LAW_NEOHOOKE) return fail(ctx, NLS_E_ARG, "the lambda mode applies to the Neo-Hooke law");
  if (mode != NLS_LAMBDA_PRINTED && mode != NLS_LAMBDA_PLANE_STRESS) return fail(ctx, NLS_E_ARG, "unknown lambda mode");
  if (mode != c.lambda_mode) c.is_setup = false;
  c.lambda_mode = mode;
  return NLS_OK;
}

int nls_set_coefficients(nls_ctx* ctx, const double* k_elem, const double* f_elem) {
  if (!ctx || !ctx->c.have_material) return fail(ctx, NLS_E_ARG, "set the material first");
  Context& c = ctx->c;
  if (c.law != NLS_LAW_DIFFUSION) return fail(ctx, NLS_E_ARG, "k_elem / f_elem apply to the diffusion law only");
  for (const double* a : {k_elem, f_elem})
    if (a)
      for (int64_t e = 0; e < c.n_elems; ++e)
        if (!std::isfinite(a[e])) return fail(ctx, NLS_E_ARG, "non-finite coefficient");
  if (k_elem)
    for (int64_t e = 0; e < c.n_elems; ++e)
      if (!(k_elem[e] > 0.0)) return fail(ctx, NLS_E_ARG, "k must be positive");
  c.k_elem.clear();
  c.f_elem.clear();
  if (k_elem) c.k_elem.assign(k_elem, k_elem + c.n_elems);
  if (f_elem) c.f_elem.assign(f_elem, f_elem + c.n_elems);
  if (!c.is_setup) return NLS_OK;
  nls::build_fext(c);
  if (!c.dev) return NLS_OK;  // host-only setup
  const int st = nls::device_set_coefficients(c);
  if (st != NLS_OK) return fail(ctx, st, c.last_error.c_str());
  return NLS_OK;
}

int nls_set_partition(nls_ctx* ctx, int32_t n_sub, const int32_t* elem_to_sub, int32_t overlap) {
  if (!ctx || !ctx->c.have_mesh) return fail(ctx, NLS_E_ARG, "set the mesh first");
  if (n_sub <= 0 || !elem_to_sub) return fail(ctx, NLS_E_ARG, "bad partition");
  if (overlap < 1) return fail(ctx, NLS_E_ARG, "overlap must be at least one element layer");
  Context& c = ctx->c;
  c.elem_to_sub.assign(elem_to_sub, elem_to_sub + c.n_elems);
  std::vector<int64_t> cnt(n_sub, 0);
  for (int32_t s : c.elem_to_sub) {
    if (s < 0 || s >= n_sub) return fail(ctx, NLS_E_ARG, "subdomain id out of range");
    cnt[s] += 1;
  }
  for (int64_t k : cnt)
    if (k == 0) return fail(ctx, NLS_E_ARG, "empty subdomain");
  c.n_sub = n_sub;
  c.overlap = overlap;
  c.have_partition = true;
  c.is_setup = false;
  return NLS_OK;
}

int nls_set_coarse(nls_ctx* ctx, int kind) {
  if (!ctx) return NLS_E_ARG;
  if (kind != NLS_COARSE_NONE && kind != NLS_COARSE_RGDSW) return fail(ctx, NLS_E_ARG, "unknown coarse space");
  ctx->c.coarse_kind = kind;
  ctx->c.is_setup = false;
  return NLS_OK;
}

int nls_set_options(nls_ctx* ctx, const nls_options* o) {
  if (!ctx || !o) return NLS_E_ARG;
  if (o->coupling < 0 || o->coupling > 2) return fail(ctx, NLS_E_ARG, "unknown coupling");
  if (o->local_precision < 0 || o->local_precision > 1 || o->coarse_precision < 0 || o->coarse_precision > 1)
    return fail(ctx, NLS_E_ARG, "unknown precision");
  if (o->load_steps < 1 || o->gmres_restart < 1 || o->gmres_maxit < 1 || o->inner_maxit < 0 || o->ls_trials < 1)
    return fail(ctx, NLS_E_ARG, "bad iteration limits");
  if (o->threads_per_block != 0 && (o->threads_per_block < 64 || o->threads_per_block > 256 || o->threads_per_block % 32))
    return fail(ctx, NLS_E_ARG, "threads_per_block must be 0 or a multiple of 32 in [64, 256]");
  if ((o->cuda_graphs != 0 && o->cuda_graphs != 1) || (o->autotune != 0 && o->autotune != 1) ||
      (o->coarse_reuse != 0 && o->coarse_reuse != 1) || (o->local_reuse != 0 && o->local_reuse != 1))
    return fail(ctx, NLS_E_ARG, "cuda_graphs, coarse_reuse, local_reuse and autotune must be 0 or 1");
  if (o->l2_prefetch < 0 || o->l2_prefetch > 64) return fail(ctx, NLS_E_ARG, "l2_prefetch must be in [0, 64]");
  if (o->outer_backtrack != 0 && o->outer_backtrack != 1) return fail(ctx, NLS_E_ARG, "outer_backtrack must be 0 or 1");
  if (o->coarse_rebuild != 0 && o->coarse_rebuild != 1) return fail(ctx, NLS_E_ARG, "coarse_rebuild must be 0 or 1");
  if (o->coarse_factor < NLS_COARSE_FACTOR_AUTO || o->coarse_factor > NLS_COARSE_FACTOR_TILES)
    return fail(ctx, NLS_E_ARG, "unknown coarse_factor");
  if (ctx->c.is_setup && (o->local_precision != ctx->c.opt.local_precision ||
                          o->coarse_precision != ctx->c.opt.coarse_precision ||
                          o->coarse_factor != ctx->c.opt.coarse_factor))
    return fail(ctx, NLS_E_ARG, "the factor precisions and the coarse factorization are fixed by nls_setup; set them before it");
  ctx->c.opt = *o;
  nls::options_changed(ctx->c);
  return NLS_OK;
}

int nls_get_options(const nls_ctx* ctx, nls_options* o) {
  if (!ctx || !o) return NLS_E_ARG;
  *o = ctx->c.opt;
  return NLS_OK;
}

namespace {
int setup_impl(nls_ctx* ctx, bool with_device) {
  if (!ctx) return NLS_E_ARG;
  Context& c = ctx->c;
  if (!c.have_mesh || !c.have_material || !c.have_partition) return fail(ctx, NLS_E_ARG, "mesh, material and partition are required");
  // Dirichlet data: whole nodes only
  const int nd = c.ndof;
  c.N = c.n_nodes * nd;
  c.dirichlet_node.assign(c.n_nodes, 0);
  c.ubc.assign(c.N, 0.0);
  std::vector<uint8_t> fixed(c.N, 0);
  for (size_t k = 0; k < c.pending_dirichlet_dofs.size(); ++k) {
    int64_t g = c.pending_dirichlet_dofs[k];
    if (g < 0 || g >= c.N) return fail(ctx, NLS_E_ARG, "Dirichlet dof out of range");
    fixed[g] = 1;
    c.ubc[g] = c.pending_dirichlet_vals[k];
  }
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    int cnt = 0;
    for (int d = 0; d < nd; ++d) cnt += fixed[v * nd + d];
    if (cnt != 0 && cnt != nd) return fail(ctx, NLS_E_UNSUPPORTED, "all components of a Dirichlet node must be fixed together");
    c.dirichlet_node[v] = cnt ? 1 : 0;
  }
  if (!c.tr_edges.empty() && c.law != NLS_LAW_NEOHOOKE) return fail(ctx, NLS_E_UNSUPPORTED, "traction applies to the Neo-Hooke law");
  if (c.coarse_kind == NLS_COARSE_NONE && c.opt.coupling != NLS_COUPLING_ONE)
    return fail(ctx, NLS_E_ARG, "additive and hybrid couplings need a coarse space");
  try {
    nls::device_free(c);
    c.is_setup = false;
    c.host_ready = false;
    int st = nls::build_setup(c);
    if (st != NLS_OK) return st;
    c.host_ready = true;
    if (with_device) {
      st = nls::device_setup(c);
      if (st != NLS_OK) return st;
      c.is_setup = true;
    }
  } catch (const std::bad_alloc&) {
    return fail(ctx, NLS_E_NOMEM, "host allocation failed during setup");
  } catch (const std::exception& ex) {
    return fail(ctx, NLS_E_ARG, ex.what());
  }
  return NLS_OK;
}
}  // namespace

int nls_setup(nls_ctx* ctx) { return setup_impl(ctx, true); }
int nls_setup_host(nls_ctx* ctx) { return setup_impl(ctx, false); }

int nls_solve(nls_ctx* ctx, double* u, int u_is_device, nls_report* rep) {
  if (!ctx || !u) return NLS_E_ARG;
  if (!ctx->c.is_setup) return fail(ctx, NLS_E_ARG, "nls_setup has not run");
  return nls::solve(ctx->c, u, u_is_device, rep);
}

int nls_get_sizes(const nls_ctx* ctx, nls_sizes* o) {
  if (!ctx || !o) return NLS_E_ARG;
  const Context& c = ctx->c;
  if (!c.host_ready) return NLS_E_ARG;
  std::memset(o, 0, sizeof(*o));
  o->n_nodes = c.n_nodes;
  o->n_dofs = c.N;
  o->n_elems = c.n_elems;
  o->ndof = c.ndof;
  o->n_sub = c.n_sub;
  o->n_coarse_nodes = c.cs.n_nodes;
  o->n_coarse_dofs = c.cs.N0;
  o->total_local_dofs = c.ov.total_n;
  o->total_overlap_elems = (int64_t)c.ov.elem_gid.size();
  o->max_local_dofs = c.ov.max_n;
  o->max_half_band = c.ov.max_b;
  o->coarse_half_band = c.cs.b0;
  o->device_bytes = c.device_bytes;
  o->total_factor_entries = c.ov.total_factor;
  o->total_local_nnz = c.ov.total_nnz;
  o->total_table_dofs = c.ov.total_nt;
  o->factor_bytes = (c.opt.local_precision == NLS_PREC_FP32_IR) ? 4 : 8;
  o->total_solve_entries = 0;
  const int64_t bs = o->factor_bytes == 4 ? 32 : 16;
  o->lu_flops = 0.0;
  o->solve_flops = 0.0;
  for (const nls::SubMeta& m : c.ov.meta) {
    o->total_solve_entries += ((m.n + bs - 1) / bs) * (2 * bs * bs + 2 * (int64_t)m.b * bs);
    for (int64_t k = 0; k < m.n; ++k) {
      const double lim = (double)std::min<int64_t>(m.b, m.n - 1 - k);
      o->lu_flops += lim + 2.0 * lim * lim;
    }
    o->solve_flops += 2.0 * (double)((m.n + bs - 1) / bs) * (2 * bs * bs + 2 * (double)m.b * bs);
  }
  return NLS_OK;
}

int nls_get_kernel_stats(const nls_ctx* ctx, int32_t cap, nls_kernel_stat* out, int32_t* n_out) {
  if (!ctx || !n_out) return NLS_E_ARG;
  return nls::kernel_stats(ctx->c, cap, out, n_out);
}

int nls_get_tuning(const nls_ctx* ctx, nls_tuning* out) {
  if (!ctx || !out) return NLS_E_ARG;
  if (!ctx->c.is_setup) return NLS_E_ARG;
  return nls::get_tuning(ctx->c, out);
}

int nls_local_corrections_noalloc(nls_ctx* ctx, const double* x, double* Fx, int32_t* its, int32_t* status,
                                  double load) {
  if (!ctx || !x || !Fx) return NLS_E_ARG;
  return nls::local_corrections_noalloc(ctx->c, x, Fx, its, status, load);
}

int nls_guess_attach(nls_ctx* ctx, nls_guess_net* net, int32_t mode) {
  if (!ctx) return NLS_E_ARG;
  return nls::guess_attach(ctx->c, net, mode);
}

int nls_guess_set_smoothing(nls_ctx* ctx, int32_t sweeps, double omega) {
  if (!ctx) return NLS_E_ARG;
  return nls::guess_set_smoothing(ctx->c, sweeps, omega);
}

int nls_guess_features(nls_ctx* ctx, const double* x, double load, float* features_out) {
  if (!ctx || !ctx->c.is_setup || !x || !features_out) return NLS_E_ARG;
  return nls::guess_features(ctx->c, x, load, features_out);
}

int nls_guess_decode(nls_ctx* ctx, const double* x, double load, const float* Y, double* guess_out) {
  if (!ctx || !ctx->c.is_setup || !x || !Y || !guess_out) return NLS_E_ARG;
  return nls::guess_decode(ctx->c, x, load, Y, guess_out);
}

int nls_guess_smooth(nls_ctx* ctx, const double* x, double load, const double* w, double* w_out) {
  if (!ctx || !ctx->c.is_setup || !x || !w || !w_out) return NLS_E_ARG;
  return nls::guess_smooth(ctx->c, x, load, w, w_out);
}

int nls_guess_counts(nls_ctx* ctx, int64_t* proposed, int64_t* accepted) {
  if (!ctx) return NLS_E_ARG;
  return nls::guess_counts(ctx->c, proposed, accepted);
}

int nls_reset_kernel_stats(nls_ctx* ctx) {
  if (!ctx) return NLS_E_ARG;
  nls::reset_kernel_stats(ctx->c);
  return NLS_OK;
}

int nls_get_local_dofs(const nls_ctx* ctx, int32_t sub, int64_t cap, int64_t* dofs, uint8_t* owned, int64_t* n_out) {
  if (!ctx || !ctx->c.host_ready || sub < 0 || sub >= ctx->c.n_sub) return NLS_E_ARG;
  const Context& c = ctx->c;
  const nls::SubMeta& m = c.ov.meta[sub];
  if (n_out) *n_out = m.n;
  if (!dofs) return NLS_OK;
  if (cap < m.n) return NLS_E_ARG;
  for (int a = 0; a < m.n; ++a) {
    dofs[a] = (int64_t)c.ov.tnode_gid[m.tnode_off + a / c.ndof] * c.ndof + a % c.ndof;
    if (owned) owned[a] = c.ov.owned[m.vec_off + a];
  }
  return NLS_OK;
}

int nls_get_overlap_elems(const nls_ctx* ctx, int32_t sub, int64_t cap, int32_t* elems, int64_t* n_out) {
  if (!ctx || !ctx->c.host_ready || sub < 0 || sub >= ctx->c.n_sub) return NLS_E_ARG;
  const Context& c = ctx->c;
  int64_t o0 = c.ov.overlap_sorted_off[sub], o1 = c.ov.overlap_sorted_off[sub + 1];
  if (n_out) *n_out = o1 - o0;
  if (!elems) return NLS_OK;
  if (cap < o1 - o0) return NLS_E_ARG;
  std::memcpy(elems, c.ov.overlap_sorted_elems.data() + o0, (o1 - o0) * sizeof(int32_t));
  return NLS_OK;
}

int nls_get_owners(const nls_ctx* ctx, int32_t* owners) {
  if (!ctx || !ctx->c.host_ready || !owners) return NLS_E_ARG;
  std::memcpy(owners, ctx->c.owner.data(), ctx->c.owner.size() * sizeof(int32_t));
  return NLS_OK;
}

int nls_get_coarse_nodes(const nls_ctx* ctx, int32_t* first) {
  if (!ctx || !ctx->c.host_ready || !first) return NLS_E_ARG;
  std::memcpy(first, ctx->c.cs.first_node.data(), ctx->c.cs.first_node.size() * sizeof(int32_t));
  return NLS_OK;
}

int nls_get_coarse_basis(const nls_ctx* ctx, double* P0) {
  if (!ctx || !ctx->c.is_setup || !P0) return NLS_E_ARG;
  return nls::get_coarse_basis(ctx->c, P0);
}

int nls_get_coarse_matrix(const nls_ctx* ctx, double* A0) {
  if (!ctx || !ctx->c.is_setup || !A0) return NLS_E_ARG;
  return nls::get_coarse_matrix(ctx->c, A0);
}

int nls_band_solve(int device, int32_t n, int32_t b, const double* band, const double* rhs, double* x,
                   int32_t precision, int32_t method, double* factors_out) {
  return nls::band_solve(device, n, b, band, rhs, x, precision, method, factors_out);
}

int nls_eval_F(nls_ctx* ctx, const double* u, double* F, int is_dev, double load) {
  if (!ctx || !ctx->c.is_setup || !u || !F) return NLS_E_ARG;
  return nls::eval_F(ctx->c, u, F, is_dev, load);
}

int nls_eval_Fx(nls_ctx* ctx, const double* u, double* Fx, int is_dev, double load, int32_t* its, int32_t* st) {
  if (!ctx || !ctx->c.is_setup || !u || !Fx) return NLS_E_ARG;
  return nls::eval_Fx(ctx->c, u, Fx, is_dev, load, its, st);
}

int nls_apply_tangent(nls_ctx* ctx, const double* v, double* y, int is_dev) {
  if (!ctx || !ctx->c.is_setup || !v || !y) return NLS_E_ARG;
  return nls::apply_tangent(ctx->c, v, y, is_dev);
}

int nls_get_local_states(nls_ctx* ctx, double* w, int is_dev) {
  if (!ctx || !ctx->c.is_setup || !w) return NLS_E_ARG;
  return nls::get_local_states(ctx->c, w, is_dev);
}

}  // extern "C"
