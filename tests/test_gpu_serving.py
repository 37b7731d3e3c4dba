"""GPU test of the continuous-batching server: every request's result is the same when it is
served in the mix (batched with other requests, other frequencies running concurrently) as
when it is solved alone, within the mixed-precision tolerance; and the mix really happened."""
import numpy as np
import pytest

from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_served_results_equal_standalone_solves():
    from paper_1801_08655_gb300 import build, hz, serving
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = W.small_problem(20, 4, 3, seed=5, R=1)
    omegas = [p.omega, 1.15 * p.omega]
    srv = serving.Server(p.m, omegas, p.npml, p.C, 3, max_cols=8, max_workers=2)
    rng = np.random.default_rng(17)
    n, lo, hi = p.n, p.npml, p.n - p.npml
    reqs = []
    for i in range(14):
        R = int(rng.integers(1, 7))
        src = np.stack([rng.integers(lo, hi, R), rng.integers(lo, hi, R), rng.integers(lo, hi, R)], axis=1)
        reqs.append(serving.Request(i, int(rng.integers(0, 2)), src, t_arrival=0.01 * i))
    wall = srv.serve(reqs)
    assert not srv.errors, srv.errors
    assert all(r.t_done is not None and r.status == 0 for r in reqs)
    assert srv.max_requests_per_batch >= 2          # requests were batched together
    st = serving.latency_stats(reqs)
    assert 0 < st["p50_s"] <= st["p99_s"] <= wall + 1e-6
    for r in reqs:
        s = srv.primaries[r.omega_idx]
        f = torch.zeros((r.R, n, n, n), dtype=torch.complex128, device="cuda")
        for k, (z, y, x) in enumerate(r.sources):
            f[k, z, y, x] = 1.0
        alone, _, _ = s.solve(f, srv.opts)
        d = float(torch.linalg.vector_norm(alone - r.result) / torch.linalg.vector_norm(alone))
        assert d < 1e-6, (r.rid, d)
    srv.close()
