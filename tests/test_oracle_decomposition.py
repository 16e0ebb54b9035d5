"""Pins of the oracle's overlapping decomposition and coarse space against hand-derived facts.

* Eq. 8: sum_i P~_i R_i = I, checked entry by entry.
* Regular box partitions, worked out by hand on the SW-NE triangulation with the
  node-sharing overlap rule: with one layer the local unknowns of box [x0, x1] x [y0, y1]
  (node indices) are exactly the free nodes of that closed box; with two layers they are the
  free nodes of [x0-1, x1+1] x [y0-1, y1+1] except its top-left and bottom-right corner
  nodes (the corner triangles that would reach them are not node-neighbours of the box).
* RGDSW on 4x4 boxes: the coarse nodes are the 9 interior cross points; with inverse-distance
  weights on straight interface edges the basis is the linear ramp between the two ends,
  including edges that end on the Dirichlet boundary (the paper's modification); the basis
  sums to one away from Dirichlet ends; the interior values are discrete-harmonic.
"""
import numpy as np
import pytest

from oracle import coarse, decomposition as dec, fem
from paper_2410_24138_gb300 import inputs as I


def _box_problem(n, nb, overlap, law="diff"):
    if law == "diff":
        return I.diffusion_problem(n, I.box_partition(n, nb, nb), nb * nb, overlap)
    return I.neohooke_problem(n, I.box_partition(n, nb, nb), nb * nb, overlap, traction_max=1.0)


@pytest.mark.parametrize("law", ["diff", "nh"])
@pytest.mark.parametrize("overlap", [1, 2])
def test_partition_of_unity(overlap, law):
    p = _box_problem(16, 3, overlap, law)
    subs, own = dec.decompose(p)
    N = p.n_nodes * p.ndof
    S = np.zeros((N, N))
    for s in subs:
        for a, g in enumerate(s.dofs):
            if s.owned[a]:
                S[g, g] += 1.0
    free = fem.free_mask(p)
    np.testing.assert_array_equal(np.diag(S)[free], 1.0)
    np.testing.assert_array_equal(np.diag(S)[~free], 0.0)


def test_c1_local_unknowns_closed_form():
    p = I.diffusion_c1()
    subs, own = dec.decompose(p)
    m = 65
    for s in subs:
        bx, by = s.index % 4, s.index // 4
        expect = [j * m + i for j in range(16 * by, 16 * by + 17) for i in range(16 * bx, 16 * bx + 17)
                  if 0 < i < 64 and 0 < j < 64]
        np.testing.assert_array_equal(s.dofs, np.array(sorted(expect)))
        assert s.n <= 289


def test_two_layer_unknowns_closed_form():
    n, nb = 24, 3
    p = _box_problem(n, nb, 2)
    subs, _ = dec.decompose(p)
    m = n + 1
    w = n // nb
    for s in subs:
        bx, by = s.index % nb, s.index // nb
        x0, x1, y0, y1 = w * bx, w * (bx + 1), w * by, w * (by + 1)
        expect = [j * m + i for j in range(y0 - 1, y1 + 2) for i in range(x0 - 1, x1 + 2)
                  if 0 < i < n and 0 < j < n and (i, j) != (x0 - 1, y1 + 1) and (i, j) != (x1 + 1, y0 - 1)]
        np.testing.assert_array_equal(s.dofs, np.array(sorted(expect)))


def test_owner_is_min_adjacent_box():
    n, nb = 12, 3
    p = _box_problem(n, nb, 1)
    _, own = dec.decompose(p)
    w = n // nb
    m = n + 1
    for j in range(m):
        for i in range(m):
            cells = [(ci, cj) for ci in (i - 1, i) for cj in (j - 1, j) if 0 <= ci < n and 0 <= cj < n]
            assert own[j * m + i] == min((cj // w) * nb + ci // w for ci, cj in cells)


def _c1_coarse():
    p = I.diffusion_c1()
    star = dec.node_star(p.conn, p.n_nodes)
    K0 = fem.global_jacobian(fem.Model(p), np.zeros(p.n_nodes))
    return p, coarse.rgdsw_coarse_space(p, star, K0), K0


def test_c1_coarse_nodes_are_cross_points():
    p, cs, _ = _c1_coarse()
    assert cs.P0.shape == (p.n_nodes, 9)
    pts = [int(c[0]) for c in cs.comps]
    assert all(len(c) == 1 for c in cs.comps)
    assert pts == sorted(65 * (16 * b) + 16 * a for b in (1, 2, 3) for a in (1, 2, 3))


def test_c1_interface_values_are_linear_ramps():
    p, cs, _ = _c1_coarse()
    P0 = cs.P0.toarray()
    m = 65
    # vertical edge x = 16 between the cross point (16, 16) (coarse 0) and the Dirichlet end (16, 0)
    for y in range(1, 16):
        np.testing.assert_allclose(P0[y * m + 16, 0], y / 16.0, rtol=1e-14)
    # horizontal edge y = 16 between cross points (16, 16) and (32, 16) (coarse 0 and 1)
    for x in range(17, 32):
        np.testing.assert_allclose(P0[16 * m + x, 0], (32 - x) / 16.0, rtol=1e-14)
        np.testing.assert_allclose(P0[16 * m + x, 1], (x - 16) / 16.0, rtol=1e-14)


def test_c1_basis_sums_to_one_away_from_dirichlet():
    p, cs, K0 = _c1_coarse()
    total = np.asarray(cs.P0.sum(axis=1)).ravel()
    m = 65
    # the central box [16, 48]^2 has no Dirichlet ancestors anywhere on or inside it
    for j in range(16, 49):
        for i in range(16, 49):
            np.testing.assert_allclose(total[j * m + i], 1.0, rtol=1e-12)


def test_c1_basis_is_discrete_harmonic():
    p, cs, K0 = _c1_coarse()
    sets = coarse.subdomain_sets(p, dec.node_star(p.conn, p.n_nodes))
    interior = np.array([v for v in range(p.n_nodes) if len(sets[v]) == 1 and v not in set(p.dirichlet_nodes.tolist())])
    res = (K0 @ cs.P0)[interior].toarray()
    assert np.max(np.abs(res)) < 1e-12


def test_elasticity_coarse_contains_translations():
    n, nb = 16, 4
    p = I.neohooke_problem(n, I.box_partition(n, nb, nb), nb * nb, 1, traction_max=1.0)
    p.dirichlet_nodes = I.boundary_nodes(n)
    star = dec.node_star(p.conn, p.n_nodes)
    K0 = fem.global_jacobian(fem.Model(p), np.zeros(p.n_nodes * 2))
    cs = coarse.rgdsw_coarse_space(p, star, K0)
    assert cs.P0.shape[1] == 3 * 9
    P0 = cs.P0.toarray()
    m = n + 1
    inner = [j * m + i for j in range(4, 13) for i in range(4, 13)]
    for comp in (0, 1):
        s = P0[:, comp::3].sum(axis=1)
        np.testing.assert_allclose(s[2 * np.array(inner) + comp], 1.0, rtol=1e-11)
        np.testing.assert_allclose(s[2 * np.array(inner) + 1 - comp], 0.0, atol=1e-11)
