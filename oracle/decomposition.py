"""Overlapping element subdomains and the operators R_i, P_i, P~_i (oracle, plain CPU code).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

Section 2 of the paper asks for an element-based overlapping partition built on the
dual graph of the mesh.  The paper does not spell out the construction; this oracle reads it as:

* Omega_i' = Omega_i grown by ``overlap`` layers; one layer adds every element that
  shares at least one node with the current element set.
* V_i (the unknowns of the local problem, Eq. 4) = the free dofs of the nodes whose whole
  element star lies in Omega_i'.  All other nodes touched by Omega_i' carry Dirichlet data
  taken from the current global iterate.  Local order = ascending global dof id.
  R_i restricts to V_i, P_i extends by zero.
* owner(node) = smallest id among the non-overlapping subdomains whose elements touch the
  node; P~_i (Eq. 8) extends by zero and keeps only the dofs that subdomain i owns, so
  sum_i P~_i R_i = I holds exactly.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2410_24138_gb300.inputs import Problem


def node_star(conn: np.ndarray, n_nodes: int):
    """CSR (ptr, elems) of the elements around every node, element ids ascending."""
    nen = conn.shape[1]
    nodes = conn.ravel()
    elems = np.repeat(np.arange(conn.shape[0]), nen)
    order = np.lexsort((elems, nodes))
    ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.add.at(ptr, nodes + 1, 1)
    return np.cumsum(ptr), elems[order]


def grow(elems: np.ndarray, conn: np.ndarray, star, layers: int) -> np.ndarray:
    """Add ``layers`` node-sharing layers of elements to an element set."""
    ptr, star_el = star
    cur = np.unique(elems)
    for _ in range(layers):
        nodes = np.unique(conn[cur])
        nb = np.concatenate([star_el[ptr[v]:ptr[v + 1]] for v in nodes])
        cur = np.unique(np.concatenate([cur, nb]))
    return cur


@dataclasses.dataclass
class Subdomain:
    index: int
    elems: np.ndarray        # elements of Omega_i', ascending
    tnodes: np.ndarray       # nodes touched by Omega_i', ascending
    lconn: np.ndarray        # connectivity of elems as positions in tnodes
    vnodes: np.ndarray       # nodes carrying local unknowns (star inside Omega_i', free), ascending
    dofs: np.ndarray         # global dof ids of the local unknowns, ascending  (R_i)
    tpos: np.ndarray         # position of each local unknown in the table dof vector
    owned: np.ndarray        # bool per local unknown: kept by P~_i
    tedges: np.ndarray       # traction segments with both nodes in tnodes (global segment ids)
    ledges: np.ndarray       # those segments as positions in tnodes

    @property
    def n(self) -> int:
        return self.dofs.shape[0]

    def table_dofs(self, ndof: int) -> np.ndarray:
        return (self.tnodes[:, None] * ndof + np.arange(ndof)[None, :]).ravel()


def owners(prob: Problem, star) -> np.ndarray:
    """owner(node) = min subdomain id of the elements around the node."""
    ptr, star_el = star
    sub_of = prob.elem_to_sub[star_el]
    return np.minimum.reduceat(sub_of, ptr[:-1]).astype(np.int32)


def decompose(prob: Problem, which=None):
    """Build the overlapping subdomains of a problem (all, or the ids in ``which``).

    Returns (subdomains, owner per node).
    """
    star = node_star(prob.conn, prob.n_nodes)
    ptr, star_el = star
    star_size = np.diff(ptr)
    own = owners(prob, star)
    dirichlet = np.zeros(prob.n_nodes, dtype=bool)
    dirichlet[prob.dirichlet_nodes] = True
    ndof = prob.ndof
    subs = []
    order = np.argsort(prob.elem_to_sub, kind="stable")
    bounds = np.searchsorted(prob.elem_to_sub[order], np.arange(prob.n_sub + 1))
    for i in (range(prob.n_sub) if which is None else which):
        base = order[bounds[i]:bounds[i + 1]]
        elems = grow(base, prob.conn, star, prob.overlap)
        tnodes, inv = np.unique(prob.conn[elems], return_inverse=True)
        lconn = inv.reshape(elems.shape[0], -1).astype(np.int64)
        inside = np.zeros(prob.n_nodes, dtype=np.int64)
        np.add.at(inside, prob.conn[elems].ravel(), 1)
        interior = (inside[tnodes] == star_size[tnodes]) & ~dirichlet[tnodes]
        vpos = np.nonzero(interior)[0]
        vnodes = tnodes[vpos]
        dofs = (vnodes[:, None] * ndof + np.arange(ndof)[None, :]).ravel()
        tpos = (vpos[:, None] * ndof + np.arange(ndof)[None, :]).ravel()
        owned = np.repeat(own[vnodes] == i, ndof)
        if prob.traction_edges is not None:
            in_t = np.zeros(prob.n_nodes, dtype=bool)
            in_t[tnodes] = True
            te = np.nonzero(in_t[prob.traction_edges[:, 0]] & in_t[prob.traction_edges[:, 1]])[0]
            le = np.searchsorted(tnodes, prob.traction_edges[te])
        else:
            te = np.zeros(0, dtype=np.int64)
            le = np.zeros((0, 2), dtype=np.int64)
        subs.append(Subdomain(i, elems, tnodes, lconn, vnodes, dofs, tpos, owned, te, le))
    return subs, own
