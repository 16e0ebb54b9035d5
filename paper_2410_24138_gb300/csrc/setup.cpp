// Host setup of the nonlinear Schwarz solver: overlapping element subdomains, local
// numbering, restricted-extension ownership (Section 2, Eq. 8), element colourings and CSR
// patterns for the batched device kernels, and the interface classification + interface
// values of the RGDSW coarse space (Section 2, option 2.2 with the Dirichlet-edge change).
//
// Everything here is integer or geometric bookkeeping, run once per mesh; the numerical
// parts of the coarse basis (the energy-minimising extension) run on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <stdexcept>
#include <thread>

#include "nls_internal.h"

namespace nls {

namespace {

const int P1_EDGES[3][2] = {{0, 1}, {1, 2}, {2, 0}};
const int Q1_EDGES[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}};

struct Scratch {
  std::vector<int32_t> elem_mark, node_mark, node_pos;
  std::vector<uint32_t> node_colors;
  int32_t stamp = 0;
  explicit Scratch(int64_t n_elems, int64_t n_nodes)
      : elem_mark(n_elems, 0), node_mark(n_nodes, 0), node_pos(n_nodes, -1), node_colors(n_nodes, 0) {}
};

// One subdomain's products before concatenation.
struct SubBuild {
  std::vector<int32_t> elems_sorted;   // ascending
  std::vector<int32_t> tnodes;         // V first, then B
  int nV = 0;
  std::vector<int32_t> elems;          // by colour
  std::vector<int32_t> lconn;
  std::vector<int32_t> color_ptr;
  std::vector<int32_t> rowptr, colidx, epos;
  std::vector<uint8_t> owned;
  int b = 0;
};

void build_one(const Context& c, const std::vector<int32_t>& base, int layers, bool neumann, int sub_id,
               Scratch& sc, SubBuild& out) {
  const int nen = c.nen, nd = c.ndof;
  // grow by node-sharing layers
  sc.stamp += 1;
  const int32_t st = sc.stamp;
  std::vector<int32_t> cur = base;
  for (int32_t e : cur) sc.elem_mark[e] = st;
  for (int l = 0; l < layers; ++l) {
    std::vector<int32_t> added;
    for (int32_t e : cur) {
      for (int a = 0; a < nen; ++a) {
        int32_t v = c.conn[(int64_t)e * nen + a];
        for (int64_t k = c.star_ptr[v]; k < c.star_ptr[v + 1]; ++k) {
          int32_t f = c.star_el[k];
          if (sc.elem_mark[f] != st) {
            sc.elem_mark[f] = st;
            added.push_back(f);
          }
        }
      }
    }
    cur.insert(cur.end(), added.begin(), added.end());
  }
  std::sort(cur.begin(), cur.end());
  out.elems_sorted = cur;
  // touched nodes; local unknowns = free nodes whose whole star lies in the element set
  std::vector<int32_t> touched;
  for (int32_t e : cur)
    for (int a = 0; a < nen; ++a) {
      int32_t v = c.conn[(int64_t)e * nen + a];
      if (sc.node_mark[v] != st) {
        sc.node_mark[v] = st;
        touched.push_back(v);
      }
    }
  std::sort(touched.begin(), touched.end());
  std::vector<int32_t> V, B;
  for (int32_t v : touched) {
    bool inside = !c.dirichlet_node[v];
    for (int64_t k = c.star_ptr[v]; inside && k < c.star_ptr[v + 1]; ++k)
      if (sc.elem_mark[c.star_el[k]] != st) inside = false;
    (inside ? V : B).push_back(v);
  }
  out.nV = (int)V.size();
  out.tnodes = V;
  out.tnodes.insert(out.tnodes.end(), B.begin(), B.end());
  for (size_t t = 0; t < out.tnodes.size(); ++t) sc.node_pos[out.tnodes[t]] = (int32_t)t;
  // greedy colouring in ascending element order
  std::vector<int> color(cur.size());
  int ncolor = 0;
  for (int32_t v : out.tnodes) sc.node_colors[v] = 0;
  for (size_t i = 0; i < cur.size(); ++i) {
    uint32_t used = 0;
    for (int a = 0; a < nen; ++a) used |= sc.node_colors[c.conn[(int64_t)cur[i] * nen + a]];
    int col = 0;
    while (used & (1u << col)) ++col;
    if (col >= 32) throw std::runtime_error("element colouring needs more than 32 colours");
    color[i] = col;
    ncolor = std::max(ncolor, col + 1);
    for (int a = 0; a < nen; ++a) sc.node_colors[c.conn[(int64_t)cur[i] * nen + a]] |= (1u << col);
  }
  std::vector<int> idx(cur.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return color[x] < color[y]; });
  out.elems.resize(cur.size());
  out.lconn.resize(cur.size() * nen);
  out.color_ptr.assign(ncolor + 1, 0);
  for (size_t i = 0; i < idx.size(); ++i) {
    int32_t e = cur[idx[i]];
    out.elems[i] = e;
    out.color_ptr[color[idx[i]] + 1] += 1;
    for (int a = 0; a < nen; ++a) out.lconn[i * nen + a] = sc.node_pos[c.conn[(int64_t)e * nen + a]];
  }
  for (int k = 0; k < ncolor; ++k) out.color_ptr[k + 1] += out.color_ptr[k];
  // CSR pattern: rows = local unknowns (or every table dof), columns = table dofs
  const int nT = (int)out.tnodes.size();
  const int row_nodes = neumann ? nT : out.nV;
  std::vector<std::vector<int32_t>> nbr(row_nodes);
  for (size_t i = 0; i < out.elems.size(); ++i)
    for (int a = 0; a < nen; ++a) {
      int32_t ta = out.lconn[i * nen + a];
      if (ta >= row_nodes) continue;
      for (int b2 = 0; b2 < nen; ++b2) nbr[ta].push_back(out.lconn[i * nen + b2]);
    }
  out.rowptr.assign(row_nodes * nd + 1, 0);
  out.colidx.clear();
  int bw = 0;
  for (int t = 0; t < row_nodes; ++t) {
    auto& L = nbr[t];
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    for (int da = 0; da < nd; ++da) {
      int row = t * nd + da;
      for (int32_t s : L)
        for (int db = 0; db < nd; ++db) {
          int col = s * nd + db;
          out.colidx.push_back(col);
          if (row < out.nV * nd && col < out.nV * nd) bw = std::max(bw, std::abs(col - row));
        }
      out.rowptr[row + 1] = (int32_t)out.colidx.size();
    }
  }
  out.b = bw;
  // element -> CSR positions
  const int ned = nen * nd;
  out.epos.assign(out.elems.size() * ned * ned, -1);
  for (size_t i = 0; i < out.elems.size(); ++i)
    for (int a = 0; a < nen; ++a) {
      int32_t ta = out.lconn[i * nen + a];
      if (ta >= row_nodes) continue;
      for (int da = 0; da < nd; ++da) {
        int row = ta * nd + da;
        const int32_t* b0 = out.colidx.data() + out.rowptr[row];
        const int32_t* b1 = out.colidx.data() + out.rowptr[row + 1];
        for (int bb = 0; bb < nen; ++bb)
          for (int db = 0; db < nd; ++db) {
            int col = out.lconn[i * nen + bb] * nd + db;
            const int32_t* p = std::lower_bound(b0, b1, col);
            out.epos[i * ned * ned + (a * nd + da) * ned + bb * nd + db] = (int32_t)(p - out.colidx.data());
          }
      }
    }
  out.owned.assign(out.nV * nd, 0);
  for (int t = 0; t < out.nV; ++t)
    for (int d = 0; d < nd; ++d) out.owned[t * nd + d] = (c.owner[out.tnodes[t]] == sub_id) ? 1 : 0;
}

}  // namespace

void build_local_set(Context& c, LocalSet& s, int layers, bool neumann_rows, bool keep_overlap_lists) {
  s = LocalSet();
  s.count = c.n_sub;
  s.ndof = c.ndof;
  s.nen = c.nen;
  s.neumann_rows = neumann_rows;
  std::vector<std::vector<int32_t>> base(c.n_sub);
  for (int64_t e = 0; e < c.n_elems; ++e) base[c.elem_to_sub[e]].push_back((int32_t)e);
  std::vector<SubBuild> parts(c.n_sub);
  unsigned nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  std::vector<std::string> errors(nthreads);
  for (unsigned t = 0; t < nthreads; ++t) {
    pool.emplace_back([&, t]() {
      try {
        Scratch sc(c.n_elems, c.n_nodes);
        for (int i = (int)t; i < c.n_sub; i += (int)nthreads) build_one(c, base[i], layers, neumann_rows, i, sc, parts[i]);
      } catch (const std::exception& ex) {
        errors[t] = ex.what();
      }
    });
  }
  for (auto& th : pool) th.join();
  for (auto& e : errors)
    if (!e.empty()) throw std::runtime_error(e);
  const int nd = c.ndof, ned = c.nen * c.ndof;
  s.meta.resize(c.n_sub);
  int64_t tn = 0, el = 0, co = 0, rp = 0, nz = 0, fa = 0, ve = 0, ep = 0, di = 0;
  for (int i = 0; i < c.n_sub; ++i) {
    SubBuild& p = parts[i];
    SubMeta& m = s.meta[i];
    m.nV = p.nV;
    m.nT = (int32_t)p.tnodes.size();
    m.n = p.nV * nd;
    m.nt = m.nT * nd;
    m.b = p.b;
    m.ne = (int32_t)p.elems.size();
    m.ncolor = (int32_t)p.color_ptr.size() - 1;
    m.nrows = (int32_t)p.rowptr.size() - 1;
    m.tnode_off = tn;
    m.elem_off = el;
    m.color_off = co;
    m.rowptr_off = rp;
    m.nnz_off = nz;
    m.nnz = (int64_t)p.colidx.size();
    m.factor_off = fa;
    m.vec_off = ve;
    m.epos_off = ep;
    m.dinv_off = di;
    tn += m.nT;
    el += m.ne;
    co += m.ncolor + 1;
    rp += m.nrows + 1;
    nz += m.nnz;
    fa += (int64_t)m.n * (2 * m.b + 1);
    ve += m.n;
    ep += (int64_t)m.ne * ned * ned;
    di += packed_solve_entries(m.n, m.b);
    s.max_n = std::max(s.max_n, m.n);
    s.max_nt = std::max(s.max_nt, m.nt);
    s.max_b = std::max(s.max_b, m.b);
    s.max_ne = std::max(s.max_ne, m.ne);
    s.max_nrows = std::max(s.max_nrows, m.nrows);
    s.tnode_gid.insert(s.tnode_gid.end(), p.tnodes.begin(), p.tnodes.end());
    s.elem_gid.insert(s.elem_gid.end(), p.elems.begin(), p.elems.end());
    s.lconn.insert(s.lconn.end(), p.lconn.begin(), p.lconn.end());
    s.color_ptr.insert(s.color_ptr.end(), p.color_ptr.begin(), p.color_ptr.end());
    s.rowptr.insert(s.rowptr.end(), p.rowptr.begin(), p.rowptr.end());
    s.colidx.insert(s.colidx.end(), p.colidx.begin(), p.colidx.end());
    s.epos.insert(s.epos.end(), p.epos.begin(), p.epos.end());
    s.owned.insert(s.owned.end(), p.owned.begin(), p.owned.end());
    if (keep_overlap_lists) {
      s.overlap_sorted_off.push_back((int64_t)s.overlap_sorted_elems.size());
      s.overlap_sorted_elems.insert(s.overlap_sorted_elems.end(), p.elems_sorted.begin(), p.elems_sorted.end());
    }
  }
  if (keep_overlap_lists) s.overlap_sorted_off.push_back((int64_t)s.overlap_sorted_elems.size());
  s.total_n = ve;
  s.total_nt = tn * nd;
  s.total_nnz = nz;
  s.total_factor = fa;
  s.total_epos = ep;
  s.total_dinv = di;
}

namespace {

// ---- global structures: colouring, CSR pattern, geometry, external load -------------------

void build_global(Context& c) {
  const int nen = c.nen, nd = c.ndof, ned = nen * nd;
  // greedy colouring of all elements
  std::vector<uint32_t> node_colors(c.n_nodes, 0);
  std::vector<int> color(c.n_elems);
  int ncolor = 0;
  for (int64_t e = 0; e < c.n_elems; ++e) {
    uint32_t used = 0;
    for (int a = 0; a < nen; ++a) used |= node_colors[c.conn[e * nen + a]];
    int col = 0;
    while (used & (1u << col)) ++col;
    if (col >= 32) throw std::runtime_error("global element colouring needs more than 32 colours");
    color[e] = col;
    ncolor = std::max(ncolor, col + 1);
    for (int a = 0; a < nen; ++a) node_colors[c.conn[e * nen + a]] |= (1u << col);
  }
  c.g_color_ptr.assign(ncolor + 1, 0);
  for (int64_t e = 0; e < c.n_elems; ++e) c.g_color_ptr[color[e] + 1] += 1;
  for (int k = 0; k < ncolor; ++k) c.g_color_ptr[k + 1] += c.g_color_ptr[k];
  c.g_elem.assign(c.n_elems, 0);
  {
    std::vector<int32_t> fill(c.g_color_ptr.begin(), c.g_color_ptr.end() - 1);
    for (int64_t e = 0; e < c.n_elems; ++e) c.g_elem[fill[color[e]]++] = (int32_t)e;
  }
  // global CSR pattern of DF (all dofs)
  c.g_rowptr.assign(c.N + 1, 0);
  c.g_col.clear();
  std::vector<int32_t> nb;
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    nb.clear();
    for (int64_t k = c.star_ptr[v]; k < c.star_ptr[v + 1]; ++k)
      for (int a = 0; a < nen; ++a) nb.push_back(c.conn[(int64_t)c.star_el[k] * nen + a]);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int da = 0; da < nd; ++da) {
      for (int32_t s : nb)
        for (int db = 0; db < nd; ++db) c.g_col.push_back(s * nd + db);
      c.g_rowptr[v * nd + da + 1] = (int32_t)c.g_col.size();
    }
  }
  if (c.g_col.size() > (size_t)INT32_MAX) throw std::runtime_error("global Jacobian too large for 32-bit positions");
  c.g_epos.assign((size_t)c.n_elems * ned * ned, 0);
  for (int64_t e = 0; e < c.n_elems; ++e)
    for (int a = 0; a < nen; ++a)
      for (int da = 0; da < nd; ++da) {
        int64_t row = (int64_t)c.conn[e * nen + a] * nd + da;
        const int32_t* b0 = c.g_col.data() + c.g_rowptr[row];
        const int32_t* b1 = c.g_col.data() + c.g_rowptr[row + 1];
        for (int bb = 0; bb < nen; ++bb)
          for (int db = 0; db < nd; ++db) {
            int32_t col = c.conn[e * nen + bb] * nd + db;
            c.g_epos[(size_t)e * ned * ned + (a * nd + da) * ned + bb * nd + db] =
                (int32_t)(std::lower_bound(b0, b1, col) - c.g_col.data());
          }
      }
  // element geometry
  if (c.elem_type == NLS_P1_TRI) {
    c.geom_stride = 8;  // G (3 x 2), area, pad
    c.geom.assign(c.n_elems * 8, 0.0);
    for (int64_t e = 0; e < c.n_elems; ++e) {
      const double* p0 = &c.xy[2 * c.conn[e * 3 + 0]];
      const double* p1 = &c.xy[2 * c.conn[e * 3 + 1]];
      const double* p2 = &c.xy[2 * c.conn[e * 3 + 2]];
      double d1x = p1[0] - p0[0], d1y = p1[1] - p0[1], d2x = p2[0] - p0[0], d2y = p2[1] - p0[1];
      double det = d1x * d2y - d1y * d2x;
      double g1x = d2y / det, g1y = -d2x / det, g2x = -d1y / det, g2y = d1x / det;
      double* g = &c.geom[e * 8];
      g[0] = -(g1x + g2x); g[1] = -(g1y + g2y);
      g[2] = g1x; g[3] = g1y; g[4] = g2x; g[5] = g2y;
      g[6] = 0.5 * det;
      g[7] = 0.0;
    }
  } else {
    c.geom_stride = 40;  // per Gauss point: dN/dX (4 x 2) and weight * det(dX/dxi)
    c.geom.assign(c.n_elems * 40, 0.0);
    const double gp = 1.0 / std::sqrt(3.0);
    const double pts[4][2] = {{-gp, -gp}, {gp, -gp}, {gp, gp}, {-gp, gp}};
    const double cr[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    for (int64_t e = 0; e < c.n_elems; ++e) {
      for (int q = 0; q < 4; ++q) {
        double xi = pts[q][0], eta = pts[q][1];
        double dN[4][2];
        for (int a = 0; a < 4; ++a) {
          dN[a][0] = 0.25 * cr[a][0] * (1.0 + eta * cr[a][1]);
          dN[a][1] = 0.25 * cr[a][1] * (1.0 + xi * cr[a][0]);
        }
        double J00 = 0, J01 = 0, J10 = 0, J11 = 0;
        for (int a = 0; a < 4; ++a) {
          const double* X = &c.xy[2 * c.conn[e * 4 + a]];
          J00 += X[0] * dN[a][0]; J01 += X[0] * dN[a][1];
          J10 += X[1] * dN[a][0]; J11 += X[1] * dN[a][1];
        }
        double det = J00 * J11 - J01 * J10;
        double i00 = J11 / det, i01 = -J01 / det, i10 = -J10 / det, i11 = J00 / det;
        double* g = &c.geom[e * 40 + q * 10];
        for (int a = 0; a < 4; ++a) {
          g[2 * a + 0] = dN[a][0] * i00 + dN[a][1] * i10;
          g[2 * a + 1] = dN[a][0] * i01 + dN[a][1] * i11;
        }
        g[8] = det;  // Gauss weight 1
        g[9] = 0.0;
      }
    }
  }
  build_fext(c);
}


// ---- RGDSW interface classification and interface values -----------------------------------

struct UnionFind {
  std::vector<int32_t> p;
  explicit UnionFind(int64_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int32_t find(int32_t x) {
    while (p[x] != x) x = p[x] = p[p[x]];
    return x;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

bool subset_of(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  return std::includes(b.begin(), b.end(), a.begin(), a.end());
}

void build_coarse(Context& c) {
  Coarse& cs = c.cs;
  cs = Coarse();
  const int nd = c.ndof, nen = c.nen;
  // S(x)
  std::vector<std::vector<int32_t>> S(c.n_nodes);
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    auto& s = S[v];
    for (int64_t k = c.star_ptr[v]; k < c.star_ptr[v + 1]; ++k) s.push_back(c.elem_to_sub[c.star_el[k]]);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
  }
  // interface nodes grouped by (S, kind), components through mesh edges
  std::map<std::pair<std::vector<int32_t>, int>, int32_t> key_of;
  std::vector<int32_t> key(c.n_nodes, -1);
  for (int64_t v = 0; v < c.n_nodes; ++v)
    if (S[v].size() >= 2) {
      auto k = std::make_pair(S[v], (int)c.dirichlet_node[v]);
      auto it = key_of.find(k);
      if (it == key_of.end()) it = key_of.emplace(k, (int32_t)key_of.size()).first;
      key[v] = it->second;
    }
  UnionFind uf(c.n_nodes);
  const int ne_edges = (c.elem_type == NLS_P1_TRI) ? 3 : 4;
  for (int64_t e = 0; e < c.n_elems; ++e)
    for (int k = 0; k < ne_edges; ++k) {
      int a = (c.elem_type == NLS_P1_TRI) ? P1_EDGES[k][0] : Q1_EDGES[k][0];
      int b = (c.elem_type == NLS_P1_TRI) ? P1_EDGES[k][1] : Q1_EDGES[k][1];
      int32_t va = c.conn[e * nen + a], vb = c.conn[e * nen + b];
      if (key[va] >= 0 && key[va] == key[vb]) uf.unite(va, vb);
    }
  std::map<int32_t, std::vector<int32_t>> comp_nodes;  // root -> nodes (ascending)
  for (int64_t v = 0; v < c.n_nodes; ++v)
    if (key[v] >= 0) comp_nodes[uf.find((int32_t)v)].push_back((int32_t)v);
  struct Comp {
    std::vector<int32_t> nodes;
    std::vector<int32_t> set;
    bool dirichlet;
  };
  std::vector<Comp> free_c, dir_c;
  for (auto& kv : comp_nodes) {
    Comp cp{kv.second, S[kv.second[0]], c.dirichlet_node[kv.second[0]] != 0};
    (cp.dirichlet ? dir_c : free_c).push_back(cp);
  }
  std::vector<std::vector<int32_t>> free_by_sub(c.n_sub), dir_by_sub(c.n_sub);
  for (size_t i = 0; i < free_c.size(); ++i)
    for (int32_t j : free_c[i].set) free_by_sub[j].push_back((int32_t)i);
  for (size_t i = 0; i < dir_c.size(); ++i)
    for (int32_t j : dir_c[i].set) dir_by_sub[j].push_back((int32_t)i);
  std::vector<int32_t> coarse;  // indices into free_c
  for (size_t i = 0; i < free_c.size(); ++i) {
    bool dominated = false;
    for (int32_t d : free_by_sub[free_c[i].set[0]])
      if (free_c[d].set.size() > free_c[i].set.size() && subset_of(free_c[i].set, free_c[d].set)) {
        dominated = true;
        break;
      }
    if (!dominated) coarse.push_back((int32_t)i);
  }
  std::sort(coarse.begin(), coarse.end(), [&](int32_t a, int32_t b) { return free_c[a].nodes[0] < free_c[b].nodes[0]; });
  cs.n_nodes = (int)coarse.size();
  const int modes = (nd == 1) ? 1 : 3;
  cs.N0 = cs.n_nodes * modes;
  std::vector<int32_t> coarse_of_free(free_c.size(), -1);
  for (size_t ci = 0; ci < coarse.size(); ++ci) {
    coarse_of_free[coarse[ci]] = (int32_t)ci;
    cs.first_node.push_back(free_c[coarse[ci]].nodes[0]);
  }
  std::vector<std::vector<int32_t>> coarse_by_sub(c.n_sub);
  for (size_t ci = 0; ci < coarse.size(); ++ci)
    for (int32_t j : free_c[coarse[ci]].set) coarse_by_sub[j].push_back((int32_t)ci);
  std::vector<double> cx(cs.n_nodes, 0.0), cy(cs.n_nodes, 0.0);
  for (int ci = 0; ci < cs.n_nodes; ++ci) {
    for (int32_t v : free_c[coarse[ci]].nodes) {
      cx[ci] += c.xy[2 * v];
      cy[ci] += c.xy[2 * v + 1];
    }
    cx[ci] /= free_c[coarse[ci]].nodes.size();
    cy[ci] /= free_c[coarse[ci]].nodes.size();
  }
  std::vector<int32_t> in_coarse(c.n_nodes, -1);
  for (int ci = 0; ci < cs.n_nodes; ++ci)
    for (int32_t v : free_c[coarse[ci]].nodes) in_coarse[v] = ci;
  auto mindist = [&](const std::vector<int32_t>& nodes, int64_t v) {
    double best = INFINITY;
    for (int32_t w : nodes) best = std::min(best, std::hypot(c.xy[2 * w] - c.xy[2 * v], c.xy[2 * w + 1] - c.xy[2 * v + 1]));
    return best;
  };
  // phi on Gamma per node: list of (coarse node, value)
  std::vector<std::vector<std::pair<int32_t, double>>> phi(c.n_nodes);
  for (int64_t v = 0; v < c.n_nodes; ++v) {
    if (S[v].size() < 2 || c.dirichlet_node[v]) continue;
    if (in_coarse[v] >= 0) {
      phi[v].push_back({in_coarse[v], 1.0});
      continue;
    }
    std::vector<std::pair<int32_t, double>> inv;
    double total = 0.0;
    for (int32_t ci : coarse_by_sub[S[v][0]])
      if (subset_of(S[v], free_c[coarse[ci]].set)) {
        double w = 1.0 / mindist(free_c[coarse[ci]].nodes, v);
        inv.push_back({ci, w});
        total += w;
      }
    for (int32_t di : dir_by_sub[S[v][0]])
      if (subset_of(S[v], dir_c[di].set)) total += 1.0 / mindist(dir_c[di].nodes, v);
    std::sort(inv.begin(), inv.end());
    for (auto& pr : inv) phi[v].push_back({pr.first, pr.second / total});
  }
  // coarse dofs per non-overlapping subdomain: every coarse function nonzero on its table
  const LocalSet& s = c.nov;
  cs.cj_ptr.assign(c.n_sub + 1, 0);
  cs.cj_col.clear();
  cs.phi_off.assign(c.n_sub + 1, 0);
  for (int j = 0; j < c.n_sub; ++j) {
    const SubMeta& m = s.meta[j];
    std::vector<int32_t> cols;
    for (int t = m.nV; t < m.nT; ++t)
      for (auto& pr : phi[s.tnode_gid[m.tnode_off + t]])
        for (int k = 0; k < modes; ++k) cols.push_back(pr.first * modes + k);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    cs.cj_col.insert(cs.cj_col.end(), cols.begin(), cols.end());
    cs.cj_ptr[j + 1] = (int32_t)cs.cj_col.size();
    cs.max_nc = std::max(cs.max_nc, (int)cols.size());
    cs.phi_off[j + 1] = cs.phi_off[j] + (int64_t)m.nt * (int64_t)cols.size();
  }
  cs.phi_total = cs.phi_off[c.n_sub];
  cs.phi_host.assign(cs.phi_total, 0.0);
  // Gamma rows of Phi_j
  for (int j = 0; j < c.n_sub; ++j) {
    const SubMeta& m = s.meta[j];
    const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
    const int32_t* cols = cs.cj_col.data() + cs.cj_ptr[j];
    for (int t = m.nV; t < m.nT; ++t) {
      int32_t v = s.tnode_gid[m.tnode_off + t];
      for (auto& pr : phi[v]) {
        int ci = pr.first;
        double val = pr.second;
        for (int k = 0; k < modes; ++k) {
          int col = ci * modes + k;
          int lc = (int)(std::lower_bound(cols, cols + nc, col) - cols);
          if (nd == 1) {
            cs.phi_host[cs.phi_off[j] + (int64_t)t * nc + lc] = val;
          } else {
            double x = c.xy[2 * v] - cx[ci], y = c.xy[2 * v + 1] - cy[ci];
            double z0 = (k == 0) ? 1.0 : (k == 1) ? 0.0 : -y;
            double z1 = (k == 0) ? 0.0 : (k == 1) ? 1.0 : x;
            cs.phi_host[cs.phi_off[j] + (int64_t)(t * 2 + 0) * nc + lc] = val * z0;
            cs.phi_host[cs.phi_off[j] + (int64_t)(t * 2 + 1) * nc + lc] = val * z1;
          }
        }
      }
    }
  }
  // P_0 as CSR over global dofs; values come from Phi blocks (p0_src)
  // every free node lies in the table of the subdomain(s) containing it; interior nodes in exactly one
  std::vector<int64_t> src_row(c.N, -1);   // Phi row index (offset of row start) per dof
  std::vector<int32_t> src_sub(c.N, -1);
  for (int j = 0; j < c.n_sub; ++j) {
    const SubMeta& m = s.meta[j];
    const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
    for (int t = 0; t < m.nT; ++t) {
      int32_t v = s.tnode_gid[m.tnode_off + t];
      if (c.dirichlet_node[v]) continue;
      for (int d = 0; d < nd; ++d) {
        int64_t g = (int64_t)v * nd + d;
        if (src_sub[g] < 0) {
          src_sub[g] = j;
          src_row[g] = cs.phi_off[j] + (int64_t)(t * nd + d) * nc;
        }
      }
    }
  }
  cs.p0_rowptr.assign(c.N + 1, 0);
  for (int64_t v = 0; v < c.n_nodes; ++v)
    for (int d = 0; d < nd; ++d) {
      int64_t g = v * nd + d;
      if (!c.dirichlet_node[v] && src_sub[g] >= 0) {
        int j = src_sub[g];
        const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
        const int32_t* cols = cs.cj_col.data() + cs.cj_ptr[j];
        // Gamma node: only the coarse functions with a nonzero interface value (all modes)
        if (S[v].size() >= 2) {
          for (auto& pr : phi[v])
            for (int k = 0; k < modes; ++k) {
              int col = pr.first * modes + k;
              int lc = (int)(std::lower_bound(cols, cols + nc, col) - cols);
              cs.p0_col.push_back(col);
              cs.p0_src.push_back(src_row[g] + lc);
            }
        } else {
          for (int lc = 0; lc < nc; ++lc) {
            cs.p0_col.push_back(cols[lc]);
            cs.p0_src.push_back(src_row[g] + lc);
          }
        }
      }
      cs.p0_rowptr[g + 1] = (int32_t)cs.p0_col.size();
    }
  // transpose
  std::vector<int32_t> cnt(cs.N0 + 1, 0);
  for (int32_t col : cs.p0_col) cnt[col + 1] += 1;
  for (int k = 0; k < cs.N0; ++k) cnt[k + 1] += cnt[k];
  cs.p0t_rowptr = cnt;
  cs.p0t_col.assign(cs.p0_col.size(), 0);
  cs.p0t_src.assign(cs.p0_col.size(), 0);
  {
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t g = 0; g < c.N; ++g)
      for (int32_t k = cs.p0_rowptr[g]; k < cs.p0_rowptr[g + 1]; ++k) {
        int32_t pos = fill[cs.p0_col[k]]++;
        cs.p0t_col[pos] = (int32_t)g;
        cs.p0t_src[pos] = k;
      }
  }
  // A_0 band structure and the per-subdomain block contributions
  int b0 = 0;
  cs.blk_off.assign(c.n_sub + 1, 0);
  for (int j = 0; j < c.n_sub; ++j) {
    const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
    const int32_t* cols = cs.cj_col.data() + cs.cj_ptr[j];
    if (nc) b0 = std::max(b0, cols[nc - 1] - cols[0]);
    cs.blk_off[j + 1] = cs.blk_off[j] + (int64_t)nc * nc;
  }
  cs.blk_total = cs.blk_off[c.n_sub];
  cs.b0 = b0;
  const int64_t W = 2 * b0 + 1;
  // two passes (count, fill) over the subdomain blocks, in subdomain order
  cs.a0_ptr.assign((size_t)cs.N0 * W + 1, 0);
  for (int j = 0; j < c.n_sub; ++j) {
    const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
    const int32_t* cols = cs.cj_col.data() + cs.cj_ptr[j];
    for (int a = 0; a < nc; ++a)
      for (int b2 = 0; b2 < nc; ++b2) cs.a0_ptr[(size_t)cols[a] * W + (cols[b2] - cols[a] + b0) + 1] += 1;
  }
  for (size_t e = 0; e + 1 < cs.a0_ptr.size(); ++e) cs.a0_ptr[e + 1] += cs.a0_ptr[e];
  cs.a0_src.assign(cs.a0_ptr.back(), 0);
  {
    std::vector<int32_t> fill(cs.a0_ptr.begin(), cs.a0_ptr.end() - 1);
    for (int j = 0; j < c.n_sub; ++j) {
      const int nc = cs.cj_ptr[j + 1] - cs.cj_ptr[j];
      const int32_t* cols = cs.cj_col.data() + cs.cj_ptr[j];
      for (int a = 0; a < nc; ++a)
        for (int b2 = 0; b2 < nc; ++b2)
          cs.a0_src[fill[(size_t)cols[a] * W + (cols[b2] - cols[a] + b0)]++] = cs.blk_off[j] + (int64_t)a * nc + b2;
    }
  }
}

}  // namespace

int build_setup(Context& c) {
  const int nd = c.ndof;
  c.N = c.n_nodes * nd;
  c.free_dof.assign(c.N, 1);
  for (int64_t v = 0; v < c.n_nodes; ++v)
    if (c.dirichlet_node[v])
      for (int d = 0; d < nd; ++d) c.free_dof[v * nd + d] = 0;
  // node stars, ascending element ids
  c.star_ptr.assign(c.n_nodes + 1, 0);
  for (int64_t e = 0; e < c.n_elems; ++e)
    for (int a = 0; a < c.nen; ++a) c.star_ptr[c.conn[e * c.nen + a] + 1] += 1;
  for (int64_t v = 0; v < c.n_nodes; ++v) c.star_ptr[v + 1] += c.star_ptr[v];
  c.star_el.assign(c.star_ptr[c.n_nodes], 0);
  {
    std::vector<int64_t> fill(c.star_ptr.begin(), c.star_ptr.end() - 1);
    for (int64_t e = 0; e < c.n_elems; ++e)
      for (int a = 0; a < c.nen; ++a) c.star_el[fill[c.conn[e * c.nen + a]]++] = (int32_t)e;
  }
  // owners
  c.owner.assign(c.n_nodes, INT32_MAX);
  for (int64_t v = 0; v < c.n_nodes; ++v)
    for (int64_t k = c.star_ptr[v]; k < c.star_ptr[v + 1]; ++k)
      c.owner[v] = std::min(c.owner[v], c.elem_to_sub[c.star_el[k]]);
  build_local_set(c, c.ov, c.overlap, false, true);
  build_global(c);
  if (c.coarse_kind == NLS_COARSE_RGDSW) {
    build_local_set(c, c.nov, 0, true, false);
    build_coarse(c);
  }
  return NLS_OK;
}

// External load at load factor 1: the source f of Eq. 1 (midpoint-rule lumping per triangle)
// and the traction of Eq. 2 (two-point rule per edge); zero on Dirichlet dofs.
void build_fext(Context& c) {
  c.fext.assign(c.N, 0.0);
  if (c.law == NLS_LAW_DIFFUSION) {
    for (int64_t e = 0; e < c.n_elems; ++e) {
      double f = c.f_elem.empty() ? 1.0 : c.f_elem[e];
      double a3 = c.geom[e * 8 + 6] / 3.0;
      for (int a = 0; a < 3; ++a) c.fext[c.conn[e * 3 + a]] += f * a3;
    }
  }
  if (c.law == NLS_LAW_NEOHOOKE && !c.f_vol.empty()) {
    // int_e f N_a dA by 2 x 2 Gauss: N_a and det J are bilinear, so the rule is exact
    const double g = 1.0 / std::sqrt(3.0);
    const double gp[4][2] = {{-g, -g}, {g, -g}, {g, g}, {-g, g}};
    const double sa[4] = {-1, 1, 1, -1}, ta[4] = {-1, -1, 1, 1};  // reference corners, counter-clockwise
    for (int64_t e = 0; e < c.n_elems; ++e) {
      const int32_t* cn = &c.conn[e * 4];
      double w[4] = {0, 0, 0, 0};
      for (const auto& q : gp) {
        double J[2][2] = {{0, 0}, {0, 0}};
        for (int a = 0; a < 4; ++a) {
          const double dxi = 0.25 * sa[a] * (1 + ta[a] * q[1]), deta = 0.25 * ta[a] * (1 + sa[a] * q[0]);
          for (int i = 0; i < 2; ++i) {
            J[i][0] += c.xy[2 * cn[a] + i] * dxi;
            J[i][1] += c.xy[2 * cn[a] + i] * deta;
          }
        }
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        for (int a = 0; a < 4; ++a) w[a] += 0.25 * (1 + sa[a] * q[0]) * (1 + ta[a] * q[1]) * det;
      }
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 2; ++d) c.fext[2 * (int64_t)cn[a] + d] += c.f_vol[2 * e + d] * w[a];
    }
  }
  for (size_t k = 0; k < c.tr_edges.size() / 2; ++k) {
    int32_t n0 = c.tr_edges[2 * k], n1 = c.tr_edges[2 * k + 1];
    double L = std::hypot(c.xy[2 * n1] - c.xy[2 * n0], c.xy[2 * n1 + 1] - c.xy[2 * n0 + 1]);
    for (int d = 0; d < 2; ++d) {
      c.fext[2 * n0 + d] += 0.5 * L * c.tr_vals[2 * k + d];
      c.fext[2 * n1 + d] += 0.5 * L * c.tr_vals[2 * k + d];
    }
  }
  for (int64_t g = 0; g < c.N; ++g)
    if (!c.free_dof[g]) c.fext[g] = 0.0;
}

}  // namespace nls
