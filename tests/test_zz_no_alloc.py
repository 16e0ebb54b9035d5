"""The allocation-free entry point nls_local_corrections_noalloc, through the C ABI.

Some callers cannot allocate device memory when they need the local corrections (a solver
step recorded into a CUDA graph, an application whose memory manager owns the GPU, a loop
that must not synchronise).  This entry point runs the batched local-Newton kernel on a
fixed scratch array compiled into the library.  Its output must match the regular entry
point nls_eval_Fx (one-level coupling) within the F_x parity tolerance of the other tests
(1e-9 relative), on two calls in a row with different points, since every call reuses the
scratch area the previous call left behind -- including as the very first call on a fresh
context, before any other entry point has run there -- and it must not change the device
memory in use.
"""
import numpy as np
import pytest

from oracle import fem
from paper_2410_24138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


def _point(p, seed):
    rng = np.random.default_rng(seed)
    return np.where(fem.free_mask(p), 0.05 * rng.random(p.n_nodes * p.ndof), 0.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_regular_entry_point(nls, precision):
    torch = pytest.importorskip("torch")
    p = I.diffusion_problem(48, I.brick_partition(48, 3, 4, 13), 12, 2)
    s = nls.make_solver(p, coupling="one", precision=precision)
    n = p.n_nodes * p.ndof
    for seed in (1, 2):  # two calls in a row, different points
        x = _point(p, seed)
        ref, ref_its, ref_st = s.eval_Fx(x)
        xd = torch.from_numpy(x).cuda()
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        its = torch.full((p.n_sub,), -1, dtype=torch.int32, device="cuda")
        st = torch.full((p.n_sub,), -1, dtype=torch.int32, device="cuda")
        s.local_corrections_noalloc(xd, out, its, st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
        np.testing.assert_array_equal(its.cpu().numpy(), ref_its)
        np.testing.assert_array_equal(st.cpu().numpy(), ref_st)


def test_noalloc_rejects_problems_beyond_its_scratch(nls):
    torch = pytest.importorskip("torch")
    p = I.diffusion_c2(n=512, per_side=16)
    s = nls.make_solver(p, coupling="one")
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(x)
    with pytest.raises(nls.NLSError) as err:
        s.local_corrections_noalloc(x, out)
    assert err.value.status == -1
    assert "scratch" in str(err.value)


def test_noalloc_first_call_on_a_fresh_context_allocates_nothing(nls):
    torch = pytest.importorskip("torch")
    p = I.diffusion_problem(40, I.brick_partition(40, 2, 3, 17), 6, 2)
    s = nls.make_solver(p, coupling="one", precision="fp32")
    n = p.n_nodes * p.ndof
    xs = [_point(p, seed) for seed in (3, 4)]
    outs = []
    for k, x in enumerate(xs):  # the first call comes straight after nls_setup
        xd = torch.from_numpy(x).cuda()
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        its = torch.full((p.n_sub,), -1, dtype=torch.int32, device="cuda")
        st = torch.full((p.n_sub,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        used, free = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        s.local_corrections_noalloc(xd, out, its, st)
        torch.cuda.synchronize()
        if k == 1:  # the first call may load the library's device code; the second must not allocate
            assert torch.cuda.memory_allocated() == used
            assert torch.cuda.mem_get_info()[0] == free
        outs.append((out.cpu().numpy(), its.cpu().numpy(), st.cpu().numpy()))
    for x, (got, its, st) in zip(xs, outs):
        ref, ref_its, ref_st = s.eval_Fx(x)
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
        np.testing.assert_array_equal(its, ref_its)
        np.testing.assert_array_equal(st, ref_st)


def test_noalloc_refuses_tensors_it_cannot_use(nls):
    torch = pytest.importorskip("torch")
    p = I.diffusion_problem(16, I.box_partition(16, 2, 2), 4, 1)
    s = nls.make_solver(p, coupling="one")
    n = p.n_nodes
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(n, dtype=torch.float32, device="cuda"),   # wrong element type
                torch.zeros(n - 1, dtype=torch.float64, device="cuda"),  # too short
                torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2]):  # not contiguous
        with pytest.raises(ValueError):
            s.local_corrections_noalloc(good, bad)
        with pytest.raises(ValueError):
            s.local_corrections_noalloc(bad, good)
    with pytest.raises(ValueError):
        s.local_corrections_noalloc(good, good, its=torch.zeros(p.n_sub, dtype=torch.int64, device="cuda"))
