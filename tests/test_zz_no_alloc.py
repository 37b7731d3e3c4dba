"""GPU test of hz_volume_residual_noalloc, the residual entry point that allocates nothing.

It exists for callers that cannot allocate device memory where they need a residual (a process
whose device memory is all held by a caching allocator, or a serving loop with a fixed memory
footprint).  It is compared through the C ABI with the allocating hz_volume_residual on calls in
a row (the later ones with more columns and different data, so stale sums in the shared fixed
scratch would show), up to its documented maximum of 1024 columns, within the FP64 tolerance of
the other residual tests; the device memory in use must not change across a call.  The file
sorts last so that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _random_volume(rng, R, n):
    return torch.from_numpy(rng.standard_normal((R, n, n, n)) + 1j * rng.standard_normal((R, n, n, n))).cuda()


def test_noalloc_residual_matches_allocating_entry_point():
    from paper_1801_08655_gb300 import build, hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 16
    p = W.small_problem(n, 3, 2, seed=12, R=3)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, 2, precision="fp64")
    rng = np.random.default_rng(4)
    for R in (2, 3, 1024):
        if R <= p.R:
            f = torch.from_numpy(p.rhs()[:R]).cuda()
        else:
            f = _random_volume(rng, R, n)
        u = _random_volume(rng, R, n)
        ref_rel, ref_r = s.volume_residual(f, u, want_r=True)
        r = torch.empty_like(f)
        torch.cuda.synchronize()
        used0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        got_rel = s.volume_residual_noalloc(f, u, r)
        torch.cuda.synchronize()
        if R != 2:   # the first call may load the kernel module; later calls must not grow memory
            assert torch.cuda.memory_allocated() == used0
            assert torch.cuda.mem_get_info()[0] == free0
        assert np.allclose(got_rel, ref_rel, rtol=1e-12, atol=0.0), (R, got_rel[:4], ref_rel[:4])
        assert float(torch.linalg.vector_norm(r - ref_r) / torch.linalg.vector_norm(ref_r)) < 1e-13
        # without the residual output as well
        got2 = s.volume_residual_noalloc(f, u)
        assert np.allclose(got2, ref_rel, rtol=1e-12, atol=0.0)
        del f, u, r, ref_r
    with pytest.raises(hz.HzError) as e:
        big = torch.zeros((1025, n, n, n), dtype=torch.complex128, device="cuda")
        s.volume_residual_noalloc(big, big)
    assert e.value.status == hz.HZ_ERR_ARG and "1024" in str(e.value)
    s.close()
