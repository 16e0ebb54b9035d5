"""The C-ABI library without a GPU: it loads, exports every symbol include/nls.h declares,
rejects bad arguments, and its host setup reproduces the oracle's integer maps bit for bit
(overlapping element sets, local numbering R_i, ownership of P~_i, coarse nodes)."""
import os
import re

import numpy as np
import pytest

from oracle import coarse as oc, decomposition as od, fem
from paper_2410_24138_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nls.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nls_[A-Za-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(nls):
    lib = nls.load()
    names = declared_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(nls.EXPORTS) == names


def test_defaults_follow_section_3(nls):
    o = nls.default_options()
    assert o.inner_rtol == 1e-5 and o.inner_atol == 1e-11
    assert o.gmres_rtol == 1e-6 and o.gmres_maxit == 1000
    assert o.outer_atol == 1e-8


def test_argument_errors(nls):
    s = nls.Solver()
    with pytest.raises(nls.NLSError):
        s.setup_host()
    p = I.diffusion_c1()
    s.set_problem(p)
    with pytest.raises(nls.NLSError):
        s.set_options(threads_per_block=100)
    with pytest.raises(nls.NLSError):
        s.set_options(load_steps=0)
    with pytest.raises(nls.NLSError):
        s.set_options(l2_prefetch=-1)
    with pytest.raises(nls.NLSError):
        s.set_options(l2_prefetch=65)
    s.set_options(l2_prefetch=0)
    bad = I.diffusion_c1()
    bad.elem_to_sub = bad.elem_to_sub.copy()
    bad.elem_to_sub[:] = 0
    bad.n_sub = 2  # subdomain 1 empty
    with pytest.raises(nls.NLSError):
        nls.make_solver(bad, coupling="one", setup="host")


def test_set_coefficients_validation(nls):
    p = I.diffusion_c1()
    s = nls.make_solver(p, coupling="one", setup="host")
    ne = p.conn.shape[0]
    s.set_coefficients(np.full(ne, 2.0), np.full(ne, 0.5))  # host-only context: accepted
    with pytest.raises(nls.NLSError):
        s.set_coefficients(np.full(ne, -1.0), None)
    bad = np.full(ne, 1.0)
    bad[3] = np.nan
    with pytest.raises(nls.NLSError):
        s.set_coefficients(None, bad)
    q = I.neohooke_problem(8, I.brick_partition(8, 2, 2, 5), 4, 1, 1.0)
    t = nls.make_solver(q, coupling="one", setup="host")
    with pytest.raises(nls.NLSError):
        t.set_coefficients(np.full(q.conn.shape[0], 1.0), None)


CASES = {
    "c1_boxes_overlap1": lambda: I.diffusion_c1(),
    "bricks_overlap2": lambda: I.diffusion_problem(48, I.brick_partition(48, 4, 4, 7), 16, 2),
    "bricks_overlap3_ragged": lambda: I.diffusion_problem(37, I.brick_partition(37, 3, 5, 9), 15, 3),
    "neohooke_bricks": lambda: I.neohooke_problem(24, I.brick_partition(24, 3, 3, 5), 9, 2, 1.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_maps_bit_exact(nls, case):
    p = CASES[case]()
    s = nls.make_solver(p, coupling="hybrid", setup="host")
    subs, own = od.decompose(p)
    np.testing.assert_array_equal(s.owners(), own)
    for sb in subs:
        d, o = s.local_dofs(sb.index)
        np.testing.assert_array_equal(d, sb.dofs)
        np.testing.assert_array_equal(o, sb.owned)
        np.testing.assert_array_equal(s.overlap_elems(sb.index), sb.elems)
    star = od.node_star(p.conn, p.n_nodes)
    K0 = fem.global_jacobian(fem.Model(p), np.zeros(p.n_nodes * p.ndof))
    cs = oc.rgdsw_coarse_space(p, star, K0)
    np.testing.assert_array_equal(s.coarse_nodes(), [int(c[0]) for c in cs.comps])
    sz = s.sizes()
    assert sz.n_coarse_dofs == cs.P0.shape[1]
    assert sz.total_local_dofs == sum(sb.n for sb in subs)


def test_full_size_c2_maps_sampled(nls):
    p = I.diffusion_c2()
    s = nls.make_solver(p, coupling="hybrid", setup="host")
    sz = s.sizes()
    assert sz.n_sub == 1024 and sz.n_dofs == 1025 * 1025
    rng = np.random.default_rng(1)
    which = sorted(rng.choice(1024, size=6, replace=False).tolist()) + [0, 1023]
    subs, own = od.decompose(p, which)
    np.testing.assert_array_equal(s.owners(), own)
    for sb in subs:
        d, o = s.local_dofs(sb.index)
        np.testing.assert_array_equal(d, sb.dofs)
        np.testing.assert_array_equal(o, sb.owned)
    # every free dof is owned by exactly one subdomain: sum_i P~_i R_i = I
    count = np.zeros(sz.n_dofs, dtype=np.int64)
    for i in range(1024):
        d, o = s.local_dofs(i)
        np.add.at(count, d[o], 1)
    free = fem.free_mask(p)
    assert np.all(count[free] == 1) and np.all(count[~free] == 0)


def test_volume_force_validation(nls):
    s = nls.Solver()
    p = I.diffusion_c1()
    s.set_problem(p)
    with pytest.raises(nls.NLSError):  # the diffusion law has no volume force
        s.set_volume_force(np.zeros((p.conn.shape[0], 2)))
    b = I.beam_problem(4, 2, 2, 4.0)
    s2 = nls.Solver()
    s2.set_problem(b)
    bad = b.f_vol.copy()
    bad[3, 1] = np.nan
    with pytest.raises(nls.NLSError):
        s2.set_volume_force(bad)
    s2.set_volume_force(None)
    s2.set_volume_force(b.f_vol)


def test_lambda_mode_validation(nls):
    s = nls.Solver()
    s.set_problem(I.diffusion_c1())
    with pytest.raises(nls.NLSError):  # the diffusion law has no Lame lambda
        s.set_lambda_mode(nls.LAMBDA_PLANE_STRESS)
    s2 = nls.Solver()
    s2.set_problem(I.neohooke_problem(8, I.brick_partition(8, 2, 2, 1), 4, 1, traction_max=1.0))
    with pytest.raises(nls.NLSError):
        s2.set_lambda_mode(7)
    s2.set_lambda_mode(nls.LAMBDA_PLANE_STRESS)
    s2.set_lambda_mode(nls.LAMBDA_PRINTED)
    # a new mode after setup invalidates it (the coarse basis and the local operators depend on it):
    # the next solve is refused before any device work
    s3 = nls.make_solver(I.neohooke_problem(8, I.brick_partition(8, 2, 2, 1), 4, 1, traction_max=1.0),
                         setup="host")
    s3.set_lambda_mode(nls.LAMBDA_PLANE_STRESS)
    with pytest.raises(nls.NLSError, match="setup"):
        s3.solve()


def test_noalloc_binding_refuses_host_arrays_before_any_launch(nls):
    """The allocation-free call passes raw device pointers to its kernel: the binding must refuse
    host arrays and CPU tensors with a ValueError, without calling into the library."""
    torch = pytest.importorskip("torch")
    p = I.diffusion_problem(16, I.box_partition(16, 2, 2), 4, 1)
    s = nls.make_solver(p, coupling="one", setup="host")
    n = p.n_nodes
    for x, out in ((np.zeros(n), np.zeros(n)),
                   (torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)),
                   (torch.zeros(n, dtype=torch.float32), torch.zeros(n, dtype=torch.float32))):
        with pytest.raises(ValueError):
            s.local_corrections_noalloc(x, out)
    s.close()
