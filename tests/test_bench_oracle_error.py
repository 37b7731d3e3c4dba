"""bench.py's accuracy report against stored oracle values (no GPU): the sampled error is exact,
and the full-grid estimate from seeded complex Gaussian sketches <w_k, u> (E|<w, e>|^2 = ||e||^2)
recovers a planted error's relative norm, here checked on a synthetic reference file of the same
format as the stored 128^3 one."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sketch_vector(N, seed, k):
    g = np.random.default_rng(seed + k).standard_normal(2 * N)
    return (g[:N] + 1j * g[N:]) / np.sqrt(2.0)


def test_samples_and_sketch_estimate(tmp_path, monkeypatch):
    rng = np.random.default_rng(0)
    R, N, K, seed = 3, 4000, 64, 77
    u_ref = rng.standard_normal((R, N)) + 1j * rng.standard_normal((R, N))
    idx = np.sort(rng.choice(N, 300, replace=False))
    sk = np.stack([u_ref @ _sketch_vector(N, seed, k) for k in range(K)], axis=1)
    path = tmp_path / "ref.npz"
    np.savez(path, idx=idx, u=u_ref[:, idx], norms=np.linalg.norm(u_ref, axis=1), sketch=sk,
             sketch_seed=seed, sketch_k=K)
    monkeypatch.setitem(bench.GOLDEN, "synthetic", str(path))
    # planted errors of relative size 1e-3, 3e-3, 1e-2 in the three columns
    rel = np.array([1e-3, 3e-3, 1e-2])
    e = rng.standard_normal((R, N)) + 1j * rng.standard_normal((R, N))
    e *= (rel * np.linalg.norm(u_ref, axis=1) / np.linalg.norm(e, axis=1))[:, None]
    u = torch.from_numpy(u_ref + e)
    out = bench.oracle_error(u, np.arange(R), "synthetic")
    exact_samples = np.linalg.norm(e[:, idx], axis=1) / np.linalg.norm(u_ref[:, idx], axis=1)
    assert out["max_rel_err_samples"] == pytest.approx(exact_samples.max(), rel=1e-12)
    # a 64-sketch estimate of the largest planted error: chi-square with 128 degrees of freedom
    assert 0.7 * rel.max() < out["max_rel_err_full_grid_sketch"] < 1.3 * rel.max()
    # the reference itself has zero error, and a subset of columns picks the matching rows
    out0 = bench.oracle_error(torch.from_numpy(u_ref[1:]), np.array([1, 2]), "synthetic")
    assert out0["max_rel_err_samples"] < 1e-15 and out0["max_rel_err_full_grid_sketch"] < 1e-12
