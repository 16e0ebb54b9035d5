"""Input and output maps of the learned initial guess, in plain FP64 numpy (oracle, CPU).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

The paper has no learned component.  This library's guess (for Eq. 1 on structured P1 meshes of
the unit square, n x n cells, node (i, j) at (i h, j h), h = 1/n) is defined as follows, and this
module writes each step out from that definition:

* Box of a subdomain: the grid rectangle [i0, i1] x [j0, j1] one node beyond the extent of its local
  unknowns (its ring of Dirichlet data from the current iterate x).
* Features (391 values): the ring data sampled at 33 equidistant points u = q/32 on each side --
  bottom (j = j0) and top (j = j1) along i, left (i = i0) and right (i = i1) along j -- by linear
  interpolation between the two grid nodes around the point; log k at the 16 x 16 points
  ((a + 1/2)/16, (b + 1/2)/16) of the box, k of the triangle containing the point (a cell is cut
  along its SW-NE diagonal; a point on the diagonal counts as in the lower triangle); the load
  factor times f of the lower triangle of the cell ((i0 + i1) // 2, (j0 + j1) // 2); the box width
  and height (i1 - i0) h, (j1 - j0) h.
* Decode: at a local unknown with box coordinates (s, t) = ((i - i0)/(i1 - i0), (j - j0)/(j1 - j0)),
  the Coons (bilinear transfinite) patch of the four sampled sides, each side read by linear
  interpolation among its 33 samples, plus the network's 32 x 32 correction, given at the points
  ((a + 1/2)/32, (b + 1/2)/32) and read bilinearly (coordinates clamped to the outermost points),
  times the target scale.
* Smoothing: `sweeps` damped Jacobi steps w <- w - omega r(w) / (d (1 + w^2)) on the local problem
  (Eq. 4), all entries at once, with r the local residual and d_a = sum over the elements e around
  node a of k_e |grad phi_a|^2 |e| (the diagonal of the Jacobian's leading term).
"""
from __future__ import annotations

import numpy as np

from oracle import fem

KSIDE, KKS, KGRID = 33, 16, 32
N_FEATURES = 4 * KSIDE + KKS * KKS + 3


def grid_indices(prob, nodes):
    m = int(round(np.sqrt(prob.n_nodes)))
    nodes = np.asarray(nodes)
    return nodes % m, nodes // m, m - 1


def ring_box(prob, unknown_nodes):
    gi, gj, _ = grid_indices(prob, unknown_nodes)
    return int(gi.min()) - 1, int(gi.max()) + 1, int(gj.min()) - 1, int(gj.max()) + 1


def side_samples(prob, box, x):
    """[4, 33]: bottom, top, left, right."""
    i0, i1, j0, j1 = box
    m = int(round(np.sqrt(prob.n_nodes)))
    node = lambda i, j: j * m + i
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
    """The 391 raw input values of one subdomain (before normalisation)."""
    box = ring_box(prob, unknown_nodes)
    i0, i1, j0, j1 = box
    n = int(round(np.sqrt(prob.n_nodes))) - 1
    h = 1.0 / n
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
    """Proposed values at the local unknowns (in the order given) from the network output Y."""
    box = ring_box(prob, unknown_nodes)
    i0, i1, j0, j1 = box
    S = side_samples(prob, box, x)
    gi, gj, _ = grid_indices(prob, unknown_nodes)
    out = np.zeros(len(unknown_nodes))
    for a in range(len(unknown_nodes)):
        s, t = (gi[a] - i0) / (i1 - i0), (gj[a] - j0) / (j1 - j0)
        out[a] = coons_samples(S, s, t) + correction(Y, s, t, tscale)
    return out


def jacobi_diagonal(prob, unknown_nodes):
    """d_a = sum_{e around a} k_e |grad phi_a|^2 |e| for P1 triangles."""
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


def smooth(local_problem, x, w, load, sweeps, omega, diag):
    """`sweeps` damped Jacobi steps on the local problem of Eq. 4 from w (x gives the ring data)."""
    w = np.array(w, dtype=float)
    for _ in range(sweeps):
        r, ok = local_problem.residual(local_problem.table(x, w), load)
        if not ok:
            break
        w = w - omega * r / (diag * (1.0 + w * w))
    return w
