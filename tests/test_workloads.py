"""The seeded synthetic workloads have the shapes, value ranges and structure their recipes state,
are reproducible, and still match the stored oracle values written from them (no GPU)."""
import math
import os

import numpy as np
import pytest

from paper_1801_08655_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def speeds(m):
    return 1.0 / np.sqrt(m)


def test_bump_workload():
    p = W.config(1)
    assert (p.n, p.npml, p.n_layers, p.R) == (24, 5, 2, 1)
    assert p.omega == pytest.approx(2 * math.pi / 8)
    c = speeds(p.m)
    assert c.max() == pytest.approx(1.3) and np.unravel_index(c.argmax(), c.shape) == (12, 12, 12)
    assert c.min() > 1.0 and tuple(p.sources[0]) == (12, 12, 12)


def test_smooth_random_workload():
    p = W.config(2)
    assert (p.n, p.npml, p.n_layers, p.R) == (64, 8, 8, 16)
    c = speeds(p.m)
    assert c.min() == pytest.approx(1.5) and c.max() == pytest.approx(4.5)
    assert p.omega == pytest.approx(2 * math.pi * 1.5 / 10)
    assert np.all(p.sources[:, 0] == 10) and len({tuple(s) for s in p.sources}) == 16
    # smooth: neighbouring cells are strongly correlated at a correlation length of 8 cells
    d = c - c.mean()
    assert np.mean(d[:, :, 1:] * d[:, :, :-1]) / np.mean(d * d) > 0.95
    assert np.array_equal(W.config(2).m, p.m)                      # seeded: reproducible


def test_layered_block_workload():
    p = W.config(3)
    assert (p.n, p.npml, p.n_layers, p.R) == (128, 10, 16, 128)
    c = speeds(p.m)
    assert set(np.round(np.unique(c), 12)) == set(np.round(np.r_[np.linspace(1.5, 4.0, 6), 4.5], 12))
    assert p.omega == pytest.approx(2 * math.pi * 1.5 / 8)
    assert np.all(p.sources[:, 0] == 12) and len({tuple(s) for s in p.sources}) == 128
    # the block sits in the middle quarter of the physical extent in x and y
    blk = np.argwhere(c == 4.5)
    nphys = 108
    for ax in (1, 2):
        frac = (blk[:, ax] - 10) / nphys
        assert frac.min() >= 0.375 and frac.max() < 0.625


def test_batched_and_serving_workloads():
    probs = W.config(4)
    assert [p.n for p in probs] == [40, 48, 64, 64, 80, 96]
    assert [p.n_layers for p in probs] == [4, 6, 8, 8, 10, 12]
    assert [p.R for p in probs] == [1, 4, 16, 32, 64, 8]
    for p in probs:
        ppw = 2 * math.pi * 1.5 / p.omega
        assert 8 - 1e-9 <= ppw <= 12 + 1e-9 and abs(ppw - round(ppw)) < 1e-9
    m, omegas = W.config(5)
    assert m.shape == (160, 160, 160)
    assert [2 * math.pi * 1.5 / w for w in omegas] == pytest.approx([8.0, 10.0, 12.0])
    reqs = W.serving_requests(160, 10, 400, rate=2.0, n_omega=3)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0) and np.mean(np.diff(t)) == pytest.approx(0.5, rel=0.2)
    for _, w, src in reqs:
        assert 0 <= w < 3 and 1 <= len(src) <= 256 and len({tuple(s) for s in src}) == len(src)


def test_stored_oracle_values_belong_to_these_workloads():
    ref3 = np.load(os.path.join(GOLDEN, "cfg3_128cube_layered_block.npz"))
    p3 = W.config(3)
    assert np.array_equal(ref3["sources"], p3.sources)
    assert ref3["u"].shape == (128, ref3["idx"].size) and ref3["relres"].max() < 1e-12
    assert ref3["idx"].min() >= 0 and ref3["idx"].max() < 128 ** 3
    for name, R in (("cfg2_64cube_smooth_samples.npz", 16), ("cfg2_64cube_density_samples.npz", 16)):
        d = np.load(os.path.join(GOLDEN, name))
        assert d["u"].shape == (R, d["idx"].size) and d["idx"].max() < 64 ** 3
        assert np.all(np.isfinite(d["u"])) and np.all(d["norms"] > 0)
