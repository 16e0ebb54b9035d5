"""RGDSW (option 2.2 with the Dirichlet-edge modification, Section 2) on a brick partition, counted
by hand, for the oracle (oracle/coarse.py) and the library's host setup (nls_setup_host).

Mesh: 12 x 12 P1 cells of the unit square (node (i, j) has id 13 j + i), homogeneous Dirichlet
data on the whole boundary.  Two bands of three bricks whose vertical cuts do not line up:
bottom band (cell rows 0..5) cut at x = 4 and 8 into subdomains 0, 1, 2; top band (rows 6..11)
cut at x = 5 and 9 into 3, 4, 5.  The horizontal interface y = 6 then carries four T-junctions,
where three subdomains meet:

  (4, 6): S = {0, 1, 3}    (5, 6): S = {1, 3, 4}    (8, 6): S = {1, 2, 4}    (9, 6): S = {2, 4, 5}

and the interface pieces between them have two-subdomain sets, each a proper subset of a
junction's set, so the coarse nodes are exactly the four junctions, in that order (ids 82, 83,
86, 87).  Ancestors and inverse-distance values (h = 1/12 cancels):

* (i, 6), i = 1..3, S = {0, 3}: coarse ancestor (4, 6) at distance 4 - i, Dirichlet ancestor
  (0, 6) (S = {0, 3}) at distance i: phi = (4 - i)^-1 / ((4 - i)^-1 + i^-1) = i / 4;
* (6, 6), (7, 6), S = {1, 4}: coarse ancestors (5, 6) and (8, 6), no Dirichlet ancestor:
  phi_(5,6) = 2/3, 1/3 and phi_(8,6) = 1/3, 2/3 (they sum to one);
* (10, 6), (11, 6), S = {2, 5}: coarse (9, 6), Dirichlet (12, 6): phi = 2/3, 1/3;
* (4, j), j = 1..5, S = {0, 1}: coarse (4, 6), Dirichlet (4, 0): phi = j / 6;
* (8, j), S = {1, 2}: coarse (8, 6): phi = j / 6;
* (5, j), j = 7..11, S = {3, 4}: coarse (5, 6), Dirichlet (5, 12): phi = (12 - j) / 6;
* (9, j), S = {4, 5}: coarse (9, 6): phi = (12 - j) / 6.
"""
import numpy as np
import pytest

from oracle import coarse, decomposition as dec, fem
from paper_2410_24138_gb300 import inputs as I

N = 12


def node(i, j):
    return j * (N + 1) + i


def brick_problem():
    cell_to_sub = np.zeros(N * N, dtype=np.int32)
    for cj in range(N):
        for ci in range(N):
            if cj < 6:
                s = 0 if ci < 4 else (1 if ci < 8 else 2)
            else:
                s = 3 if ci < 5 else (4 if ci < 9 else 5)
            cell_to_sub[cj * N + ci] = s
    return I.diffusion_problem(N, cell_to_sub, 6, 1)


EXPECTED_COARSE = [node(4, 6), node(5, 6), node(8, 6), node(9, 6)]
EXPECTED_SETS = [(0, 1, 3), (1, 3, 4), (1, 2, 4), (2, 4, 5)]


def expected_phi():
    """node -> {coarse index: value} on every free interface node, from the table above."""
    out = {}
    for k, v in enumerate(EXPECTED_COARSE):
        out[v] = {k: 1.0}
    for i in (1, 2, 3):
        out[node(i, 6)] = {0: i / 4}
    out[node(6, 6)] = {1: 2 / 3, 2: 1 / 3}
    out[node(7, 6)] = {1: 1 / 3, 2: 2 / 3}
    out[node(10, 6)] = {3: 2 / 3}
    out[node(11, 6)] = {3: 1 / 3}
    for j in range(1, 6):
        out[node(4, j)] = {0: j / 6}
        out[node(8, j)] = {2: j / 6}
    for j in range(7, 12):
        out[node(5, j)] = {1: (12 - j) / 6}
        out[node(9, j)] = {3: (12 - j) / 6}
    return out


def test_oracle_brick_t_junctions():
    p = brick_problem()
    star = dec.node_star(p.conn, p.n_nodes)
    K0 = fem.global_jacobian(fem.Model(p), np.zeros(p.n_nodes))
    cs = coarse.rgdsw_coarse_space(p, star, K0)
    assert [int(c[0]) for c in cs.comps] == EXPECTED_COARSE
    assert [tuple(s) for s in cs.comp_sets] == EXPECTED_SETS
    exp = expected_phi()
    assert sorted(cs.phi_gamma) == sorted(exp)
    for v, entries in exp.items():
        got = cs.phi_gamma[v]
        assert sorted(got) == sorted(entries), v
        for k, val in entries.items():
            assert got[k] == pytest.approx(val, rel=0, abs=1e-15), (v, k)
    # on Gamma the basis columns carry exactly these values (the extension only fills the interior)
    P0 = cs.P0.toarray()
    for v, entries in exp.items():
        row = np.zeros(len(EXPECTED_COARSE))
        for k, val in entries.items():
            row[k] = val
        np.testing.assert_allclose(P0[v], row, rtol=0, atol=1e-15)


def test_library_host_setup_finds_the_same_coarse_nodes():
    from paper_2410_24138_gb300 import build, nls
    build.build()
    s = nls.make_solver(brick_problem(), coupling="hybrid", setup="host")
    assert s.coarse_nodes().tolist() == EXPECTED_COARSE
    assert s.sizes().n_coarse_dofs == 4
    s.close()
