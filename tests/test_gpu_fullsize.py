"""Parity at the benchmark's full size, on sampled outputs.

The 1024 x 1024 diffusion workload (1.05M dofs, 1024 uneven subdomains, overlap 2) and the
512 x 512 one with a log-normal k field (0.26M dofs, 256 subdomains) run through
the same batched kernels and the autotuned launch configuration the benchmark times (FP32
factors + FP64 refinement).  The oracle cannot solve the whole problem in a test's time, but
every owned entry of F_1(u) = sum_i P~_i T_i(u) (Eq. 5) and of its tangent (Eq. 6) comes from one
subdomain's local problem, which the oracle solves on its own: six subdomains (both ends of the
numbering, the middle and three seeded picks) are compared entry by entry.  Both sides drive
their local Newton loops to 1e-14, so the bounds are those of the small-size tests: 1e-9 for
F_x, 1e-7 for the tangent (FP32 factors refined to 1e-10), and local iteration counts within
one.

The 512 x 512 Neo-Hooke workload (Eq. 2, Q1, 0.53M dofs, 256 uneven subdomains, overlap 2), and
the local path of the 2048 x 2048 one (8.4M dofs, 4096 subdomains), are checked the same way on
five subdomains, at the first load step's traction (load factor 0.2) and a smooth bending state
u_y = -0.02 x^2 with a seeded perturbation of 1e-5 (no element near inversion).  At h = 1/512 the
local residuals cannot be driven to 1e-14 (the line search stalls at the rounding floor of the
stiffness, E = 210), so both sides stop at 1e-12 relative / 1e-13 absolute; Newton's last step
takes both far below that.  Both forms run: F_x within 1e-9 in both; the tangent within 1e-9 in the
FP64 form and 1e-7 in the FP32 form, whose FP32 factors are refined to 1e-10 against the local
Jacobian assembled from FP64 element tangents -- the same bounds as for Eq. 1.  Every comparison
is also made entry by entry in the max norm, at ten times the l2 bound.

The whole pipeline at full size (hybrid coupling: coarse Newton, local solves, exact tangent in
GMRES, outer Newton) is checked on the 1024 x 1024 diffusion workload against the oracle's plain
global Newton on the same mesh (F(u) = 0 of Eq. 1 written out, sparse direct FP64 solves): both
sides are driven to ||F|| < 1e-12, and the converged solutions must agree within 1e-8 (FP64 form)
and 1e-6 (FP32 factors + refinement) relative l2, the bounds of the small-size tests.
"""
import numpy as np
import pytest

from oracle import fem, schwarz as S
from paper_2410_24138_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TIGHT = dict(inner_rtol=1e-14, inner_atol=1e-15)


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


@pytest.mark.parametrize("workload", ["c2", "c4"])
def test_full_size_sampled_local_corrections_and_tangent(nls, workload):
    # c4: the 512 x 512 learned-guess workload (log-normal k, constant f), a held-out field seed
    p = I.diffusion_c2() if workload == "c2" else I.diffusion_c4(1001)
    s = nls.make_solver(p, coupling="one", precision="fp32", autotune=1, **TIGHT)
    rng = np.random.default_rng(2410)
    free = fem.free_mask(p)
    u = np.where(free, 0.05 * rng.random(p.n_nodes), 0.0)
    v = np.where(free, rng.random(p.n_nodes), 0.0)
    Fx, its, st = s.eval_Fx(u, 1.0)
    y = s.apply_tangent(v)
    assert np.all(st == 0)
    assert s.tuning()["newton_tuned"]
    pick = sorted({0, p.n_sub // 2, p.n_sub - 1, *rng.choice(p.n_sub, 3, replace=False).tolist()})
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, **TIGHT), with_coarse=False, which=pick)
    Fo, sto = sw.evaluate(u, 1.0)
    yo = sw.tangent(sto)(v)
    for k, (lp, res) in enumerate(zip(sw.locals, sto["local"])):
        owned = lp.sub.dofs[lp.sub.owned]
        assert np.linalg.norm(Fx[owned] - Fo[owned]) <= 1e-9 * np.linalg.norm(Fo[owned])
        assert np.abs(Fx[owned] - Fo[owned]).max() <= 1e-8 * np.abs(Fo[owned]).max()
        assert np.linalg.norm(y[owned] - yo[owned]) <= 1e-7 * np.linalg.norm(yo[owned])
        assert np.abs(y[owned] - yo[owned]).max() <= 1e-6 * np.abs(yo[owned]).max()
        assert abs(int(its[pick[k]]) - res.its) <= 1


@pytest.mark.parametrize("workload,precision", [("c3", "fp64"), ("c3", "fp32"), ("c5", "fp32")])
def test_full_size_neohooke_sampled_local_corrections_and_tangent(nls, workload, precision):
    # c5: the 2048 x 2048 workload (8.4M dofs, 4096 subdomains) on its local path only
    p = I.neohooke_c3() if workload == "c3" else I.neohooke_c5()
    tight = dict(inner_rtol=1e-12, inner_atol=1e-13)
    s = nls.make_solver(p, coupling="one", precision=precision, autotune=1, **tight)
    rng = np.random.default_rng(2410)
    free = fem.free_mask(p)
    u = np.zeros(p.n_nodes * p.ndof)
    u[1::2] = -0.02 * p.xy[:, 0] ** 2
    u = np.where(free, u + 1e-5 * rng.random(u.size), 0.0)
    v = np.where(free, rng.random(u.size), 0.0)
    load = 0.2
    Fx, its, st = s.eval_Fx(u, load)
    y = s.apply_tangent(v)
    assert np.all(st == 0)
    pick = sorted({0, p.n_sub // 2, p.n_sub - 1, *rng.choice(p.n_sub, 2, replace=False).tolist()})
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, **tight), with_coarse=False, which=pick)
    Fo, sto = sw.evaluate(u, load)
    yo = sw.tangent(sto)(v)
    for k, (lp, res) in enumerate(zip(sw.locals, sto["local"])):
        assert res.status == 0
        owned = lp.sub.dofs[lp.sub.owned]
        assert np.linalg.norm(Fx[owned] - Fo[owned]) <= 1e-9 * np.linalg.norm(Fo[owned])
        assert np.abs(Fx[owned] - Fo[owned]).max() <= 1e-8 * np.abs(Fo[owned]).max()
        assert abs(int(its[pick[k]]) - res.its) <= 1
        tol = 1e-9 if precision == "fp64" else 1e-7
        assert np.linalg.norm(y[owned] - yo[owned]) <= tol * np.linalg.norm(yo[owned])
        assert np.abs(y[owned] - yo[owned]).max() <= 10 * tol * np.abs(yo[owned]).max()


def test_full_size_converged_solution_matches_oracle_plain_newton(nls):
    p = I.diffusion_c2()
    ustar, _ = S.plain_newton(p, tol=1e-12, load_steps=p.load_steps)
    F = fem.global_residual(fem.Model(p), ustar)
    assert np.linalg.norm(F) < 1e-12
    for precision, tol in (("fp64", 1e-8), ("fp32", 1e-6)):
        # local solves tight enough that their corrections still resolve ||F|| ~ 1e-12 (with the
        # default local tolerance every correction vanishes once ||F|| ~ 1e-11: F_x = 0, done)
        s = nls.make_solver(p, coupling="hybrid", precision=precision, outer_atol=1e-12, inner_atol=1e-15)
        u, rep = s.solve()
        s.close()
        assert rep.status == 0 and rep.final_residual < 1e-12, (precision, rep.final_residual)
        err = np.linalg.norm(u - ustar) / np.linalg.norm(ustar)
        assert err < tol, (precision, err)
