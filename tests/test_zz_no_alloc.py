"""GPU test of hz_volume_residual_noalloc, the residual entry point that allocates nothing.

It is compared through the C ABI with the allocating hz_volume_residual on two calls in a
row (the second with more columns and different data, so stale sums in the shared fixed
scratch would show), within the FP64 tolerance of the other residual tests.  The file sorts
last so that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_allocating_entry_point():
    from paper_1801_08655_gb300 import build, hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = W.small_problem(16, 3, 2, seed=12, R=3)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, 2, precision="fp64")
    rng = np.random.default_rng(4)
    for R in (2, 3):
        f = torch.from_numpy(p.rhs()[:R]).cuda()
        u = torch.from_numpy(rng.standard_normal((R, 16, 16, 16)) + 1j * rng.standard_normal((R, 16, 16, 16))).cuda()
        ref_rel, ref_r = s.volume_residual(f, u, want_r=True)
        r = torch.empty_like(f)
        got_rel = s.volume_residual_noalloc(f, u, r)
        torch.cuda.synchronize()
        assert np.allclose(got_rel, ref_rel, rtol=1e-12, atol=0.0), (got_rel, ref_rel)
        assert float(torch.linalg.vector_norm(r - ref_r) / torch.linalg.vector_norm(ref_r)) < 1e-13
    with pytest.raises(hz.HzError) as e:
        big = torch.zeros((1025, 16, 16, 16), dtype=torch.complex128, device="cuda")
        s.volume_residual_noalloc(big, big)
    assert e.value.status == hz.HZ_ERR_ARG and "1024" in str(e.value)
    s.close()
