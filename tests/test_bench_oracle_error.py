"""bench.py's accuracy report and clock record (no GPU): the sampled error is exact,
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


def test_clock_sampler_summary():
    """The clock record of the timed region: median SM clock under load, the maximum, and every
    throttle reason seen active (the fields of the nvidia-smi query the bench runs)."""
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.lines = [
        "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, 2060, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active",
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2065.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]
