"""Parity at the benchmark's full size, on sampled outputs.

The 1024 x 1024 diffusion workload (1.05M dofs, 1024 uneven subdomains, overlap 2) runs through
the same batched kernels and the autotuned launch configuration the benchmark times (FP32
factors + FP64 refinement).  The oracle cannot solve the whole problem in a test's time, but
every owned entry of F_1(u) = sum_i P~_i T_i(u) (Eq. 5) and of its tangent (Eq. 6) comes from one
subdomain's local problem, which the oracle solves on its own: six subdomains (both ends of the
numbering, the middle and three seeded picks) are compared entry by entry.  Both sides drive
their local Newton loops to 1e-14, so the bounds are those of the small-size tests: 1e-9 for
F_x, 1e-7 for the tangent (FP32 factors refined to 1e-10), and local iteration counts within
one.
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


def test_full_size_sampled_local_corrections_and_tangent(nls):
    p = I.diffusion_c2()
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
        assert np.linalg.norm(y[owned] - yo[owned]) <= 1e-7 * np.linalg.norm(yo[owned])
        assert abs(int(its[pick[k]]) - res.its) <= 1
