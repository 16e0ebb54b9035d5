"""RGDSW coarse space, option 2.2, with the paper's Dirichlet-edge modification (oracle, CPU).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

Section 2 of the paper uses the reduced GDSW space of Dohrmann and Widlund with
option 2.2 (inverse Euclidean distance weights on the interface), changed so that
interface edges ending at a Dirichlet boundary also get inverse-distance values
instead of the constant one.  Written out, with the readings where the paper is silent:

* S(x) = set of non-overlapping subdomains whose elements touch node x.
  Interface = nodes with |S(x)| >= 2.  Interface nodes are grouped by (S, free or
  Dirichlet) and split into mesh-edge-connected components.
* Coarse nodes = free components whose S is not a proper subset of the S of another
  free component; ordered by their smallest global node id.
* Ancestors of an interface node x = coarse components C with S(C) >= S(x) plus
  Dirichlet components D with S(D) >= S(x) (the modification: Dirichlet ends act as
  ancestors whose own basis function is dropped).
* phi_C(x) = 1 on C itself; elsewhere phi_C(x) = d(x, C)^-1 / sum_{A ancestors} d(x, A)^-1,
  with d(x, A) the distance from x to the nearest node of A.
* Interior values: the energy-minimising (discrete harmonic) extension
  phi_I = -K_II^-1 K_IG phi_G in every non-overlapping subdomain, K = DF(u^(0)).
* Elasticity: three functions per coarse node, phi_C * z with z in
  {(1, 0), (0, 1), (-(y - y_C), x - x_C)}, (x_C, y_C) the centroid of C.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

from paper_2410_24138_gb300.inputs import P1_TRI, Problem

P1_EDGE_PAIRS = ((0, 1), (1, 2), (2, 0))
Q1_EDGE_PAIRS = ((0, 1), (1, 2), (2, 3), (3, 0))


def subdomain_sets(prob: Problem, star):
    """S(x) of every node as a tuple of ascending subdomain ids."""
    ptr, star_el = star
    subs = prob.elem_to_sub[star_el]
    return [tuple(sorted(set(subs[ptr[v]:ptr[v + 1]].tolist()))) for v in range(prob.n_nodes)]


def mesh_edges(prob: Problem) -> np.ndarray:
    pairs = P1_EDGE_PAIRS if prob.elem_type == P1_TRI else Q1_EDGE_PAIRS
    e = np.concatenate([prob.conn[:, [a, b]] for a, b in pairs])
    return np.unique(np.sort(e, axis=1), axis=0)


@dataclasses.dataclass
class CoarseSpace:
    P0: sp.csr_matrix            # N x N0 basis (rows = global dofs)
    comps: list                  # node arrays of the coarse components, in coarse order
    comp_sets: list              # S of each coarse component
    phi_gamma: dict              # node -> {coarse component: value} on the interface
    interface_nodes: np.ndarray  # free interface nodes


def interface_components(prob: Problem, sets, dirichlet: np.ndarray):
    """Components of interface nodes with equal (S, kind), connected through mesh edges."""
    iface = np.array([len(s) >= 2 for s in sets])
    key_of = {}
    key_id = np.full(prob.n_nodes, -1, dtype=np.int64)
    for v in np.nonzero(iface)[0]:
        key = (sets[v], bool(dirichlet[v]))
        key_id[v] = key_of.setdefault(key, len(key_of))
    e = mesh_edges(prob)
    same = (key_id[e[:, 0]] >= 0) & (key_id[e[:, 0]] == key_id[e[:, 1]])
    e = e[same]
    g = sp.coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(prob.n_nodes, prob.n_nodes))
    _, label = csgraph.connected_components(g, directed=False)
    comps = {}
    for v in np.nonzero(iface)[0]:
        comps.setdefault(label[v], []).append(v)
    out = []
    for nodes in comps.values():
        nodes = np.array(sorted(nodes))
        out.append((nodes, sets[nodes[0]], bool(dirichlet[nodes[0]])))
    return out


def rgdsw_coarse_space(prob: Problem, star, K0: sp.csr_matrix) -> CoarseSpace:
    ndof = prob.ndof
    N = prob.n_nodes * ndof
    dirichlet = np.zeros(prob.n_nodes, dtype=bool)
    dirichlet[prob.dirichlet_nodes] = True
    sets = subdomain_sets(prob, star)
    comps = interface_components(prob, sets, dirichlet)
    free_c = [c for c in comps if not c[2]]
    dir_c = [c for c in comps if c[2]]

    # components indexed by each of their subdomains, so superset searches stay local
    by_sub = {}
    for idx, c in enumerate(free_c):
        for j in c[1]:
            by_sub.setdefault(j, []).append(idx)

    def has_proper_superset(c):
        return any(len(free_c[d][1]) > len(c[1]) and set(c[1]) <= set(free_c[d][1]) for d in by_sub[c[1][0]])

    coarse = [c for c in free_c if not has_proper_superset(c)]
    coarse.sort(key=lambda c: int(c[0][0]))
    n_coarse = len(coarse)
    xy = prob.xy
    coarse_by_sub, dir_by_sub = {}, {}
    for ci, c in enumerate(coarse):
        for j in c[1]:
            coarse_by_sub.setdefault(j, []).append(ci)
    for di, c in enumerate(dir_c):
        for j in c[1]:
            dir_by_sub.setdefault(j, []).append(di)

    # values on the interface (Gamma)
    in_comp = {}
    for ci, (nodes, _, _) in enumerate(coarse):
        for v in nodes:
            in_comp[int(v)] = ci
    phi_gamma = {}
    interface_nodes = np.array([v for v in range(prob.n_nodes) if len(sets[v]) >= 2 and not dirichlet[v]], dtype=np.int64)
    for v in interface_nodes:
        v = int(v)
        if v in in_comp:
            phi_gamma[v] = {in_comp[v]: 1.0}
            continue
        s = set(sets[v])
        first = sets[v][0]
        anc = [ci for ci in coarse_by_sub.get(first, []) if s <= set(coarse[ci][1])]
        anc_d = [di for di in dir_by_sub.get(first, []) if s <= set(dir_c[di][1])]
        inv = {ci: 1.0 / np.min(np.linalg.norm(xy[coarse[ci][0]] - xy[v], axis=1)) for ci in anc}
        total = sum(inv.values()) + sum(1.0 / np.min(np.linalg.norm(xy[dir_c[di][0]] - xy[v], axis=1)) for di in anc_d)
        phi_gamma[v] = {ci: w / total for ci, w in inv.items()}

    # coarse basis vectors on Gamma, one column per (coarse node, mode)
    n_modes = 1 if ndof == 1 else 3
    N0 = n_coarse * n_modes
    centroid = np.array([xy[nodes].mean(axis=0) for nodes, _, _ in coarse]) if n_coarse else np.zeros((0, 2))
    rows, cols, vals = [], [], []
    for v, entries in phi_gamma.items():
        for ci, phi in entries.items():
            if ndof == 1:
                rows.append(v); cols.append(ci); vals.append(phi)
            else:
                x, y = xy[v] - centroid[ci]
                for comp, mode, val in ((0, 0, 1.0), (1, 1, 1.0), (0, 2, -y), (1, 2, x)):
                    rows.append(2 * v + comp); cols.append(3 * ci + mode); vals.append(phi * val)
    PG = sp.coo_matrix((vals, (rows, cols)), shape=(N, N0)).tocsr()

    # energy-minimising extension into the interior of every non-overlapping subdomain
    interior_nodes = np.array([v for v in range(prob.n_nodes) if len(sets[v]) == 1 and not dirichlet[v]], dtype=np.int64)
    owner_of_interior = np.array([sets[v][0] for v in interior_nodes], dtype=np.int64)
    PI_blocks = []
    K0 = K0.tocsr()
    for j in range(prob.n_sub):
        nodes = interior_nodes[owner_of_interior == j]
        if nodes.size == 0:
            continue
        I = (nodes[:, None] * ndof + np.arange(ndof)[None, :]).ravel()
        KII = K0[I][:, I].tocsc()
        rhs = -(K0[I] @ PG)                        # K_IG phi_G (Gamma columns are the only nonzeros of PG)
        rhs = rhs.toarray()
        touched = np.nonzero(np.any(rhs != 0.0, axis=0))[0]
        if touched.size == 0:
            continue
        lu = spla.splu(KII)
        sol = lu.solve(rhs[:, touched])
        r_, c_ = np.nonzero(sol)
        PI_blocks.append(sp.coo_matrix((sol[r_, c_], (I[r_], touched[c_])), shape=(N, N0)))
    P0 = PG
    for b in PI_blocks:
        P0 = P0 + b.tocsr()
    return CoarseSpace(P0.tocsr(), [c[0] for c in coarse], [c[1] for c in coarse], phi_gamma, interface_nodes)
