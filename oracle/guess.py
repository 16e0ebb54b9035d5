"""Input and output maps of the learned initial guess, in plain FP64 numpy (oracle, CPU).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

The paper has no learned component.  This library's guess works on structured meshes of the unit
square, n x n cells, node (i, j) at (i h, j h), h = 1/n: P1 triangles with one unknown per node
(Eq. 1) or Q1 quadrilaterals with the two displacement components per node (Eq. 2, local unknowns
ordered node-major, component-interleaved).  It is defined as follows, and this module writes each
step out from that definition:

* Box of a subdomain: the grid rectangle [i0, i1] x [j0, j1] one node beyond the extent of its local
  unknowns, clamped to the mesh [0, n] x [0, n].  For Eq. 1 with Dirichlet data on the whole
  boundary the clamp never acts and the box sides are the subdomain's ring of Dirichlet data from the
  current iterate x; where local unknowns reach a Neumann edge (Eq. 2) that side of the box is the
  edge itself, carrying current values of x.
* Side samples: x (one component) at 33 equidistant points u = q/32 on each side -- bottom (j = j0)
  and top (j = j1) along i, left (i = i0) and right (i = i1) along j -- by linear interpolation
  between the two grid nodes around the point.
* Features, Eq. 1 (391 values): the side samples; log k at the 16 x 16 points ((a + 1/2)/16,
  (b + 1/2)/16) of the box, k of the triangle containing the point (a cell is cut along its SW-NE
  diagonal; a point on the diagonal counts as in the lower triangle); the load factor times f of the
  lower triangle of the cell ((i0 + i1) // 2, (j0 + j1) // 2); the box width and height (i1 - i0) h,
  (j1 - j0) h.
* Features, Eq. 2 (267 values): the side samples of the first and then of the second displacement
  component (2 x 132); the load factor; the box width and height.
* Decode: at a local unknown (component c) with box coordinates (s, t) = ((i - i0)/(i1 - i0),
  (j - j0)/(j1 - j0)), the Coons (bilinear transfinite) patch of component c's four sampled sides,
  each side read by linear interpolation among its 33 samples, plus the network's 32 x 32
  correction for component c (outputs c * 1024 .. c * 1024 + 1023), given at the points
  ((a + 1/2)/32, (b + 1/2)/32) and read bilinearly (coordinates clamped to the outermost points),
  times the target scale.
* Smoothing: `sweeps` damped Jacobi steps w <- w - omega r(w) / (d q(w)) on the local problem
  (Eq. 4), all entries at once, with r the local residual; Eq. 1: q = 1 + w^2 and d_a = sum over the
  elements e around node a of k_e |grad phi_a|^2 |e| (the diagonal of the Jacobian's leading term);
  Eq. 2: q = 1 and d the diagonal of the linear-elastic stiffness (the tangent at zero displacement),
  d_(a,c) = sum over elements and Gauss points of w det(J) ((lambda + 2 mu) (dN_a/dX_c)^2 +
  mu (dN_a/dX_c')^2), c' the other component.
"""
from __future__ import annotations

import numpy as np

from oracle import fem
from paper_2410_24138_gb300.inputs import LAMBDA_PLANE_STRESS

KSIDE, KKS, KGRID = 33, 16, 32
N_FEATURES = 4 * KSIDE + KKS * KKS + 3          # Eq. 1
N_FEATURES_DISP = 2 * 4 * KSIDE + 3             # Eq. 2


def grid_indices(prob, nodes):
    m = int(round(np.sqrt(prob.n_nodes)))
    nodes = np.asarray(nodes)
    return nodes % m, nodes // m, m - 1


def ring_box(prob, unknown_nodes):
    gi, gj, n = grid_indices(prob, unknown_nodes)
    return (max(int(gi.min()) - 1, 0), min(int(gi.max()) + 1, n), max(int(gj.min()) - 1, 0),
            min(int(gj.max()) + 1, n))


def side_samples(prob, box, x, comp=0):
    """[4, 33]: bottom, top, left, right, of displacement component `comp` (0 for Eq. 1)."""
    i0, i1, j0, j1 = box
    m = int(round(np.sqrt(prob.n_nodes)))
    nd = prob.ndof
    node = lambda i, j: (j * m + i) * nd + comp
    S = np.zeros((4, KSIDE))
    for q in range(KSIDE):
        u = q / (KSIDE - 1)
        fi, fj = i0 + u * (i1 - i0), j0 + u * (j1 - j0)
        ii, jj = min(int(np.floor(fi)), i1 - 1), min(int(np.floor(fj)), j1 - 1)
        wi, wj = fi - ii, fj - jj
        S[0, q] = (1 - wi) * x[node(ii, j0)] + wi * x[node(ii + 1, j0)]
        S[1, q] = (1 - wi) * x[node(ii, j1)] + wi * x[node(ii + 1, j1)]
        S[2, q] = (1 - wj) * x[node(i0, jj)] + wj * x[node(i0, jj + 1)]
        S[3, q] = (1 - wj) * x[node(i1, jj)] + wj * x[node(i1, jj + 1)]
    return S


def features(prob, unknown_nodes, x, load):
    """The raw input values of one subdomain (before normalisation): 391 for Eq. 1, 267 for Eq. 2."""
    box = ring_box(prob, unknown_nodes)
    i0, i1, j0, j1 = box
    n = int(round(np.sqrt(prob.n_nodes))) - 1
    h = 1.0 / n
    if prob.ndof == 2:
        return np.concatenate([side_samples(prob, box, x, 0).ravel(), side_samples(prob, box, x, 1).ravel(),
                               [load, (i1 - i0) * h, (j1 - j0) * h]])
    k = np.ones(prob.conn.shape[0]) if prob.k_elem is None else prob.k_elem
    f = np.ones(prob.conn.shape[0]) if prob.f_elem is None else prob.f_elem
    logk = np.zeros(KKS * KKS)
    for b in range(KKS):
        for a in range(KKS):
            fx, fy = i0 + (a + 0.5) / KKS * (i1 - i0), j0 + (b + 0.5) / KKS * (j1 - j0)
            ci, cj = min(int(fx), n - 1), min(int(fy), n - 1)
            lower = (fx - ci) >= (fy - cj)
            logk[b * KKS + a] = np.log(k[2 * (cj * n + ci) + (0 if lower else 1)])
    ci, cj = min((i0 + i1) // 2, n - 1), min((j0 + j1) // 2, n - 1)
    fval = load * f[2 * (cj * n + ci)]
    return np.concatenate([side_samples(prob, box, x).ravel(), logk, [fval, (i1 - i0) * h, (j1 - j0) * h]])


def side_value(S, side, u):
    q = u * (KSIDE - 1)
    i0 = max(0, min(KSIDE - 2, int(np.floor(q))))
    w = q - i0
    return (1 - w) * S[side, i0] + w * S[side, i0 + 1]


def coons_samples(S, s, t):
    P00, P10, P01, P11 = S[0, 0], S[0, KSIDE - 1], S[1, 0], S[1, KSIDE - 1]
    return ((1 - t) * side_value(S, 0, s) + t * side_value(S, 1, s) + (1 - s) * side_value(S, 2, t)
            + s * side_value(S, 3, t) - ((1 - s) * (1 - t) * P00 + s * (1 - t) * P10 + (1 - s) * t * P01 + s * t * P11))


def correction(Y, s, t, tscale):
    gx = min(max(s * KGRID - 0.5, 0.0), KGRID - 1.0)
    gy = min(max(t * KGRID - 0.5, 0.0), KGRID - 1.0)
    a0, b0 = min(int(gx), KGRID - 2), min(int(gy), KGRID - 2)
    wa, wb = gx - a0, gy - b0
    Yg = np.asarray(Y).reshape(KGRID, KGRID)  # [b][a]
    v = ((1 - wa) * (1 - wb) * Yg[b0, a0] + wa * (1 - wb) * Yg[b0, a0 + 1] + (1 - wa) * wb * Yg[b0 + 1, a0]
         + wa * wb * Yg[b0 + 1, a0 + 1])
    return v * tscale


def decode(prob, unknown_nodes, x, Y, tscale):
    """Proposed values at the local unknowns (nodes in the order given, components interleaved)
    from the network output Y (KGRID^2 values per component)."""
    box = ring_box(prob, unknown_nodes)
    i0, i1, j0, j1 = box
    nd = prob.ndof
    S = [side_samples(prob, box, x, c) for c in range(nd)]
    Y = np.asarray(Y)
    gi, gj, _ = grid_indices(prob, unknown_nodes)
    out = np.zeros(len(unknown_nodes) * nd)
    for a in range(len(unknown_nodes)):
        s, t = (gi[a] - i0) / (i1 - i0), (gj[a] - j0) / (j1 - j0)
        for c in range(nd):
            Yc = Y[c * KGRID * KGRID:(c + 1) * KGRID * KGRID]
            out[a * nd + c] = coons_samples(S[c], s, t) + correction(Yc, s, t, tscale)
    return out


def jacobi_diagonal(prob, unknown_nodes):
    """Eq. 1: d_a = sum_{e around a} k_e |grad phi_a|^2 |e| for P1 triangles.  Eq. 2: the diagonal of
    the linear-elastic Q1 stiffness (2 x 2 Gauss points), components interleaved."""
    if prob.ndof == 2:
        return elasticity_diagonal(prob, unknown_nodes)
    k = np.ones(prob.conn.shape[0]) if prob.k_elem is None else prob.k_elem
    pos = {int(v): a for a, v in enumerate(unknown_nodes)}
    d = np.zeros(len(unknown_nodes))
    for e, tri in enumerate(prob.conn):
        X = prob.xy[tri]
        area, G = fem.p1_gradients(X[None])
        for a in range(3):
            v = int(tri[a])
            if v in pos:
                d[pos[v]] += k[e] * area[0] * float(G[0, a] @ G[0, a])
    return d


def elasticity_diagonal(prob, unknown_nodes):
    mu, lam = fem.lame(prob.young, prob.poisson, prob.lambda_mode == LAMBDA_PLANE_STRESS)
    pos = {int(v): a for a, v in enumerate(unknown_nodes)}
    d = np.zeros(2 * len(unknown_nodes))
    g = 1.0 / np.sqrt(3.0)
    for e, quad in enumerate(prob.conn):
        X = prob.xy[quad]
        for xi, eta in ((-g, -g), (g, -g), (g, g), (-g, g)):
            dN = fem.q1_shape_derivatives(xi, eta)  # [4, 2], d/dxi, d/deta
            J = X.T @ dN                            # dX/dxi
            G = dN @ np.linalg.inv(J)               # dN/dX
            wdet = np.linalg.det(J)
            for a in range(4):
                v = int(quad[a])
                if v in pos:
                    for c in range(2):
                        d[2 * pos[v] + c] += wdet * ((lam + 2 * mu) * G[a, c] ** 2 + mu * G[a, 1 - c] ** 2)
    return d


def smooth(local_problem, x, w, load, sweeps, omega, diag):
    """`sweeps` damped Jacobi steps on the local problem of Eq. 4 from w (x gives the ring data)."""
    w = np.array(w, dtype=float)
    scalar = local_problem.model.ndof == 1
    for _ in range(sweeps):
        r, ok = local_problem.residual(local_problem.table(x, w), load)
        if not ok:
            break
        w = w - omega * r / (diag * ((1.0 + w * w) if scalar else 1.0))
    return w
