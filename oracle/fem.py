"""Finite-element residuals and tangents of the two model problems (oracle, FP64, CPU).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.  Parity of every function here is pinned by ``tests/test_oracle_fem.py``.

* Eq. 1, nonlinear diffusion  -div(k (1 + u^2) grad u) = f,  P1 triangles.
  Element residual  r_a = int_T k (1 + u^2) grad u . grad phi_a  -  int_T f phi_a.
  The integrand (1 + u^2) is quadratic on a triangle, so the three-edge-midpoint rule
  (weights |T|/3) integrates it exactly; f is constant per element.
* Eq. 2, compressible Neo-Hooke, Q1 quadrilaterals, 2 dofs per node,
  P(F) = mu (F - F^-T) + lambda ln(det F) F^-T  with mu = E / (2 (1 + nu)) and
  lambda = E nu / ((1 + nu)(1 - 2 nu)).  (The printed formula has "E/(1(1+nu))" and
  "ln(det(F) F^-T)"; both are read as this standard law.)  2x2 Gauss quadrature; dead
  load traction on boundary segments by 2-point Gauss (exact for a constant traction) and a
  dead-load volume force f_vol, constant per element, by 2x2 Gauss (exact: N_a det J is at
  most quadratic in each reference coordinate).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from paper_2410_24138_gb300.inputs import LAMBDA_PLANE_STRESS, LAW_DIFFUSION, LAW_NEOHOOKE, Problem


def lame(young: float, poisson: float, plane_stress: bool = False):
    """(mu, lambda) of the compressible Neo-Hooke law, Eq. 2: lambda as printed, or (plane_stress)
    reduced so that the out-of-plane stress of the linearised law vanishes, lambda* = 2 mu lambda /
    (lambda + 2 mu)."""
    mu = young / (2.0 * (1.0 + poisson))
    lam = young * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson))
    if plane_stress:
        lam = 2.0 * mu * lam / (lam + 2.0 * mu)
    return mu, lam


# ----------------------------------------------------------------------------------------------
# Eq. 1: nonlinear diffusion on P1 triangles
# ----------------------------------------------------------------------------------------------

def p1_gradients(X: np.ndarray):
    """Area and constant gradients of the three barycentric coordinates of each triangle.

    X: [E, 3, 2] vertex coordinates (counter-clockwise).  Returns (area [E], G [E, 3, 2]).
    """
    d1 = X[:, 1] - X[:, 0]
    d2 = X[:, 2] - X[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    g1 = np.stack([d2[:, 1], -d2[:, 0]], axis=1) / det[:, None]
    g2 = np.stack([-d1[:, 1], d1[:, 0]], axis=1) / det[:, None]
    g0 = -(g1 + g2)
    return 0.5 * det, np.stack([g0, g1, g2], axis=1)


P1_EDGES = ((0, 1), (1, 2), (2, 0))


def diffusion_p1(X: np.ndarray, ue: np.ndarray, k: np.ndarray, f: np.ndarray, want_jac: bool = True):
    """Element residual r [E, 3] and tangent K [E, 3, 3] (K[e, a, b] = d r_a / d u_b) of Eq. 1."""
    area, G = p1_gradients(X)
    grad_u = np.einsum("ea,eai->ei", ue, G)
    mid = np.stack([0.5 * (ue[:, a] + ue[:, b]) for a, b in P1_EDGES], axis=1)      # u at edge midpoints
    Q = area / 3.0 * np.sum(1.0 + mid * mid, axis=1)                                 # int_T (1 + u^2)
    flux = np.einsum("ei,eai->ea", grad_u, G)                                        # grad u . grad phi_a
    r = (k * Q)[:, None] * flux - (f * area / 3.0)[:, None]
    if not want_jac:
        return r, None
    # d Q / d u_b = |T|/3 * sum of the midpoint values on the two edges that touch vertex b
    dQ = np.zeros_like(ue)
    for e_idx, (a, b) in enumerate(P1_EDGES):
        dQ[:, a] += mid[:, e_idx]
        dQ[:, b] += mid[:, e_idx]
    dQ *= (area / 3.0)[:, None]
    GG = np.einsum("eai,ebi->eab", G, G)
    K = (k * Q)[:, None, None] * GG + k[:, None, None] * flux[:, :, None] * dQ[:, None, :]
    return r, K


# ----------------------------------------------------------------------------------------------
# Eq. 2: compressible Neo-Hooke on Q1 quadrilaterals
# ----------------------------------------------------------------------------------------------

_GP = 1.0 / np.sqrt(3.0)
Q1_GAUSS = np.array([[-_GP, -_GP], [_GP, -_GP], [_GP, _GP], [-_GP, _GP]])
Q1_CORNERS = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]])


def q1_shape_derivatives(xi: float, eta: float) -> np.ndarray:
    """d N_a / d(xi, eta) of the bilinear shape functions N_a = (1 + xi xi_a)(1 + eta eta_a) / 4."""
    return np.stack([0.25 * Q1_CORNERS[:, 0] * (1.0 + eta * Q1_CORNERS[:, 1]),
                     0.25 * Q1_CORNERS[:, 1] * (1.0 + xi * Q1_CORNERS[:, 0])], axis=1)


def neohooke_stress(Fd: np.ndarray, mu: float, lam: float):
    """First Piola-Kirchhoff stress P(F) and its tangent A_iJkL = dP_iJ / dF_kL for F [..., 2, 2]."""
    det = Fd[..., 0, 0] * Fd[..., 1, 1] - Fd[..., 0, 1] * Fd[..., 1, 0]
    Finv = np.empty_like(Fd)
    Finv[..., 0, 0] = Fd[..., 1, 1] / det
    Finv[..., 1, 1] = Fd[..., 0, 0] / det
    Finv[..., 0, 1] = -Fd[..., 0, 1] / det
    Finv[..., 1, 0] = -Fd[..., 1, 0] / det
    FinvT = np.swapaxes(Finv, -1, -2)
    lnJ = np.log(det)
    P = mu * (Fd - FinvT) + (lam * lnJ)[..., None, None] * FinvT
    eye = np.eye(2)
    A = (mu * np.einsum("ik,JL->iJkL", eye, eye)
         + lam * np.einsum("...Ji,...Lk->...iJkL", Finv, Finv)
         + (mu - lam * lnJ)[..., None, None, None, None] * np.einsum("...Jk,...Li->...iJkL", Finv, Finv))
    return P, A, det


def neohooke_q1(X: np.ndarray, ue: np.ndarray, mu: float, lam: float, want_jac: bool = True):
    """Element residual r [E, 8] (dof = 2 * node + component) and tangent K [E, 8, 8] of Eq. 2.

    Returns (r, K, min det F over the Gauss points).
    """
    E = X.shape[0]
    r = np.zeros((E, 4, 2))
    K = np.zeros((E, 4, 2, 4, 2)) if want_jac else None
    detmin = np.full(E, np.inf)
    U = ue.reshape(E, 4, 2)
    for xi, eta in Q1_GAUSS:
        dN = q1_shape_derivatives(xi, eta)                    # [4, 2]
        Jm = np.einsum("eai,aj->eij", X, dN)                  # dX_i / dxi_j
        detJm = Jm[:, 0, 0] * Jm[:, 1, 1] - Jm[:, 0, 1] * Jm[:, 1, 0]
        Jinv = np.stack([np.stack([Jm[:, 1, 1], -Jm[:, 0, 1]], 1),
                         np.stack([-Jm[:, 1, 0], Jm[:, 0, 0]], 1)], 1) / detJm[:, None, None]
        B = np.einsum("aj,eji->eai", dN, Jinv)                # dN_a / dX_i
        Fd = np.eye(2)[None] + np.einsum("eai,eaJ->eiJ", U, B)
        P, A, det = neohooke_stress(Fd, mu, lam)
        detmin = np.minimum(detmin, det)
        r += detJm[:, None, None] * np.einsum("eiJ,eaJ->eai", P, B)
        if want_jac:
            K += detJm[:, None, None, None, None] * np.einsum("eiJkL,eaJ,ebL->eaibk", A, B, B)
    return r.reshape(E, 8), (K.reshape(E, 8, 8) if want_jac else None), detmin


def q1_shape_values(xi: float, eta: float) -> np.ndarray:
    """N_a(xi, eta) = (1 + xi xi_a)(1 + eta eta_a) / 4 at the four corners a."""
    return 0.25 * (1.0 + xi * Q1_CORNERS[:, 0]) * (1.0 + eta * Q1_CORNERS[:, 1])


def volume_load(X: np.ndarray, f: np.ndarray) -> np.ndarray:
    """External force int_e f . N_a dA of a constant volume force f [E, 2] on Q1 elements X [E, 4, 2]:
    [E, 8] (dof = 2 * node + component)."""
    w = np.zeros((X.shape[0], 4))
    for xi, eta in Q1_GAUSS:
        Jm = np.einsum("eai,aj->eij", X, q1_shape_derivatives(xi, eta))
        detJm = Jm[:, 0, 0] * Jm[:, 1, 1] - Jm[:, 0, 1] * Jm[:, 1, 0]
        w += detJm[:, None] * q1_shape_values(xi, eta)[None, :]
    return (w[:, :, None] * f[:, None, :]).reshape(X.shape[0], 8)


def traction_load(Xe: np.ndarray, t: np.ndarray) -> np.ndarray:
    """External force int_edge t N_a ds on each boundary segment: [M, 4] (dof = 2 * node + comp).

    The shape functions are linear on a segment and t is constant, so each end node
    receives t * length / 2 (what 2-point Gauss gives exactly).
    """
    length = np.linalg.norm(Xe[:, 1] - Xe[:, 0], axis=1)
    half = 0.5 * length[:, None] * t
    return np.concatenate([half, half], axis=1)


# ----------------------------------------------------------------------------------------------
# element loops over arbitrary element sets, global F(u) and DF(u) of Eq. 3
# ----------------------------------------------------------------------------------------------

class Model:
    """Element terms of a problem, evaluated on any subset of its elements."""

    def __init__(self, prob: Problem):
        self.prob = prob
        self.ndof = prob.ndof
        self.nen = prob.conn.shape[1]
        n_el = prob.conn.shape[0]
        self.k = np.ones(n_el) if prob.k_elem is None else np.asarray(prob.k_elem, dtype=np.float64)
        self.f = np.ones(n_el) if prob.f_elem is None else np.asarray(prob.f_elem, dtype=np.float64)
        self.mu, self.lam = lame(prob.young, prob.poisson, prob.lambda_mode == LAMBDA_PLANE_STRESS)
        self.fvol = None if prob.f_vol is None else np.asarray(prob.f_vol, dtype=np.float64).reshape(n_el, 2)

    def element_terms(self, elems: np.ndarray, Xe: np.ndarray, ue: np.ndarray, want_jac: bool = True,
                      load: float = 1.0):
        """(r [E, nen*ndof], K [E, nen*ndof, nen*ndof] or None, ok flag) for the listed elements.

        ``load`` scales the external source f of Eq. 1 and the volume force of Eq. 2 (load stepping
        ramps every external load).
        ``ok`` is False when a Neo-Hooke element has det F <= 0 at a Gauss point.
        """
        if self.prob.law == LAW_DIFFUSION:
            r, K = diffusion_p1(Xe, ue, self.k[elems], load * self.f[elems], want_jac)
            return r, K, True
        with np.errstate(invalid="ignore", divide="ignore"):
            r, K, detmin = neohooke_q1(Xe, ue, self.mu, self.lam, want_jac)
        if self.fvol is not None:
            r = r - load * volume_load(Xe, self.fvol[elems])
        return r, K, bool(np.all(detmin > 0.0))

    def external_load(self, edges: np.ndarray, Xe: np.ndarray, load: float) -> np.ndarray:
        """Dead-load traction forces [M, 4] of the listed traction segments at load factor ``load``."""
        return traction_load(Xe, load * self.prob.traction[edges])


def element_dofs(conn: np.ndarray, ndof: int) -> np.ndarray:
    """Dof ids (node * ndof + component) of every element, node-major."""
    return (conn[:, :, None] * ndof + np.arange(ndof)[None, None, :]).reshape(conn.shape[0], -1)


def free_mask(prob: Problem) -> np.ndarray:
    mask = np.ones(prob.n_nodes * prob.ndof, dtype=bool)
    mask[prob.dirichlet_dofs()] = False
    return mask


def global_residual(model: Model, u: np.ndarray, load: float = 1.0) -> np.ndarray:
    """F(u) of Eq. 3 over all dofs at load factor ``load`` (scaling f and g_N); Dirichlet rows are zero."""
    prob = model.prob
    all_e = np.arange(prob.conn.shape[0])
    dofs = element_dofs(prob.conn, model.ndof)
    r, _, _ = model.element_terms(all_e, prob.xy[prob.conn], u[dofs], want_jac=False, load=load)
    F = np.zeros(u.shape[0])
    np.add.at(F, dofs.ravel(), r.ravel())
    if prob.traction_edges is not None:
        ed = element_dofs(prob.traction_edges, model.ndof)
        fe = model.external_load(np.arange(ed.shape[0]), prob.xy[prob.traction_edges], load)
        np.add.at(F, ed.ravel(), -fe.ravel())
    F[~free_mask(prob)] = 0.0
    return F


def global_jacobian(model: Model, u: np.ndarray) -> sp.csr_matrix:
    """DF(u) of Eq. 3 as an N x N sparse matrix over all dofs (Dirichlet rows/cols included)."""
    prob = model.prob
    all_e = np.arange(prob.conn.shape[0])
    dofs = element_dofs(prob.conn, model.ndof)
    _, K, _ = model.element_terms(all_e, prob.xy[prob.conn], u[dofs], want_jac=True)
    nd = dofs.shape[1]
    rows = np.repeat(dofs, nd, axis=1).ravel()
    cols = np.tile(dofs, (1, nd)).ravel()
    N = u.shape[0]
    return sp.coo_matrix((K.ravel(), (rows, cols)), shape=(N, N)).tocsr()
