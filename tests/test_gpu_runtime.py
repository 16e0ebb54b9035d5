"""The launch runtime around the kernels: the GMRES cycle as one CUDA graph of conditional
nodes, and the autotuner of the CTA sizes.

* The graph of a GMRES cycle launches the same kernels with the same arguments in the same order
  as plain stream launches (the Givens step runs on the device either way; in the graph it ends
  the cycle by switching off the conditional nodes of the later iterations), so the solution,
  every iteration count and the launch count must be identical bit for bit, and one cycle graph
  must have been captured.
* The autotuner only changes the CTA size of the batched local kernels, which changes the
  order of the floating-point reductions inside a subdomain: the converged solution must agree
  with the fixed choice within the FP32-factor bound of the solution parity tests (1e-6
  relative), and the choice must be one of the candidates.
* Each path converges to the oracle's solution of F(u) = 0 (Eq. 3) on the same problem.
* Swapping the coefficients k, f of Eq. 1 on a set-up context (nls_set_coefficients) gives the
  same solution, bit for bit, as a context set up for those coefficients from the start.
* Reusing the stored local factors for chord steps (local_reuse) and the previous tangent phase's
  coarse factorization (coarse_reuse) only changes how the local and coarse problems are solved
  to their stopping tests: the converged solution agrees with the fresh-Jacobian iteration within
  the FP32-path bound (1e-6) and solves F(u) = 0 of the oracle to the outer tolerance.
"""
import numpy as np
import pytest

from oracle import fem, schwarz as S
from paper_2410_24138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


def _brick():
    return I.diffusion_problem(64, I.brick_partition(64, 4, 4, 7), 16, 2)


@pytest.mark.parametrize("coupling", ["add", "hybrid"])
def test_graph_replay_is_bit_identical(nls, coupling):
    p = _brick()
    a = nls.make_solver(p, coupling=coupling, cuda_graphs=0, outer_atol=1e-12)
    ua, ra = a.solve()
    b = nls.make_solver(p, coupling=coupling, cuda_graphs=1, outer_atol=1e-12)
    ub, rb = b.solve()
    assert ra.status == 0 and rb.status == 0
    assert np.array_equal(ua, ub)
    for k in ("outer_iterations", "gmres_iterations", "subdomain_newton_steps", "coarse_newton_steps",
              "kernel_launches"):
        assert getattr(ra, k) == getattr(rb, k), k
    t = b.tuning()
    assert t["graphs_captured"] == 1
    assert a.tuning()["graphs_captured"] == 0
    # a second solve on the same context replays the captured graphs
    ub2, rb2 = b.solve()
    assert np.array_equal(ub, ub2) and rb2.kernel_launches == rb.kernel_launches


def test_graphs_follow_option_changes(nls):
    p = _brick()
    s = nls.make_solver(p, coupling="hybrid", outer_atol=1e-12)
    u1, r1 = s.solve()
    n1 = s.tuning()["graphs_captured"]
    s.set_options(coupling=nls.COUPLING["add"], outer_atol=1e-12)
    u2, r2 = s.solve()
    ref = nls.make_solver(p, coupling="add", cuda_graphs=0, outer_atol=1e-12)
    u3, r3 = ref.solve()
    assert n1 > 0
    assert np.array_equal(u2, u3) and r2.gmres_iterations == r3.gmres_iterations


@pytest.mark.parametrize("law", ["diffusion", "neohooke"])
def test_autotuner_choice_and_solution(nls, law):
    if law == "diffusion":
        p = _brick()
    else:
        p = I.neohooke_problem(24, I.brick_partition(24, 2, 3, 5), 6, 2, traction_max=4.0, load_steps=2)
    a = nls.make_solver(p, coupling="hybrid", outer_atol=1e-11)
    ua, ra = a.solve()
    b = nls.make_solver(p, coupling="hybrid", outer_atol=1e-11, autotune=1)
    ub, rb = b.solve()
    assert ra.status == 0 and rb.status == 0
    t = b.tuning()
    assert t["newton_tuned"] and t["apply_tuned"]
    sz = b.sizes()
    need = (32 + sz.max_half_band + 31) // 32 * 32
    assert t["newton_threads"] in (128, 256) and t["newton_threads"] >= need
    assert need <= t["apply_threads"] <= 256 and t["apply_threads"] % 32 == 0
    assert np.linalg.norm(ub - ua) <= 1e-6 * np.linalg.norm(ua)
    F = fem.global_residual(fem.Model(p), ub)
    assert np.linalg.norm(F) < 1e-8


def test_graph_path_matches_oracle_solution(nls):
    p = I.diffusion_c1()
    s = nls.make_solver(p, coupling="hybrid", precision="fp64", outer_atol=1e-12, cuda_graphs=1)
    u, rep = s.solve()
    assert s.tuning()["graphs_captured"] > 0
    uo, _ = S.plain_newton(p, tol=1e-14)
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)


def test_set_coefficients_matches_fresh_setup(nls):
    n, per = 64, 4
    k1, f1 = I.c4_elem_coefficients(7, n)
    fresh = nls.make_solver(I.diffusion_c4(7, n=n, per_side=per), coupling="hybrid", outer_atol=1e-12)
    u1, r1 = fresh.solve()
    reused = nls.make_solver(I.diffusion_c4(8, n=n, per_side=per), coupling="hybrid", outer_atol=1e-12)
    reused.solve()
    reused.set_coefficients(k1, f1)
    u2, r2 = reused.solve()
    assert r1.status == 0 and r2.status == 0
    assert np.array_equal(u1, u2)
    assert np.array_equal(fresh.coarse_basis(), reused.coarse_basis())


def test_factor_reuse_keeps_the_solution(nls):
    p = I.neohooke_problem(24, I.brick_partition(24, 2, 3, 5), 6, 2, traction_max=4.0, load_steps=2)
    a = nls.make_solver(p, coupling="hybrid", outer_atol=1e-11, local_reuse=0, coarse_reuse=0)
    ua, ra = a.solve()
    b = nls.make_solver(p, coupling="hybrid", outer_atol=1e-11, local_reuse=1, coarse_reuse=1)
    ub, rb = b.solve()
    assert ra.status == 0 and rb.status == 0
    assert ra.local_chord_steps == 0 and rb.local_chord_steps > 0
    assert np.linalg.norm(ub - ua) <= 1e-6 * np.linalg.norm(ua)
    F = fem.global_residual(fem.Model(p), ub)
    assert np.linalg.norm(F) < 1e-8


@pytest.mark.parametrize("coupling", ["one", "hybrid"])
def test_l2_prefetch_changes_no_result(nls, coupling):
    """The L2 prefetch of the triangular solves' operands is a hint: solutions and iteration
    counts are bit-identical with it off and on."""
    p = _brick()
    runs = []
    for dist in (0, 4):
        s = nls.make_solver(p, coupling=coupling, outer_atol=1e-12, l2_prefetch=dist)
        u, rep = s.solve()
        assert rep.status == 0
        runs.append((u, rep))
    (u0, r0), (u4, r4) = runs
    assert np.array_equal(u0, u4)
    for k in ("outer_iterations", "gmres_iterations", "subdomain_newton_steps", "local_chord_steps"):
        assert getattr(r0, k) == getattr(r4, k), k
