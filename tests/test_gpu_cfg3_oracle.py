"""Parity of the 128^3 headline workload with the CPU oracle (GPU).

The workload is the bench's: 128^3 layered + block medium, PML 10, 16 layers, 128 point sources,
solved in the bench's launch configuration (default autotuning, all 128 right-hand sides in one
call, GMRES to 1e-4 and FP64 defect correction to a volume residual of 1e-5) in mixed precision,
and 8 of the sources in FP64 mode.  The stored values come from the multifrontal FP64 global
direct solve of the same discrete system (tests/golden/make_golden_cfg3.py, which calls only
the oracle):
  * 512 seeded sample points per right-hand side: relative L2 error over the samples;
  * the full-grid relative L2 error estimated from 16 sketches <w_k, u> with seeded complex
    Gaussian w_k (E|<w, e>|^2 = ||e||^2), so that an error anywhere in the 2M-point grid shows;
  * the full-grid norm of every solution.
Tolerances: 1e-5 (mixed), 1e-6 (FP64), the relative-error targets of the method's two precisions.
"""
import os

import numpy as np
import pytest

from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg3_128cube_layered_block.npz")


def _sketch_vectors(N, seed, K, device):
    W_ = torch.empty((K, N), dtype=torch.complex128, device=device)
    for k in range(K):
        g = np.random.default_rng(seed + k).standard_normal(2 * N)
        W_[k] = torch.from_numpy((g[:N] + 1j * g[N:]) / np.sqrt(2.0)).to(device)
    return W_


def _check(u, ref, cols, tol, label):
    """u: (R, N) complex128 CUDA tensor of the solutions of the golden sources `cols`."""
    idx = torch.from_numpy(ref["idx"]).to(u.device)
    samples = u[:, idx].cpu().numpy()
    s_ref = ref["u"][cols]
    e_samp = np.linalg.norm(samples - s_ref, axis=1) / np.linalg.norm(s_ref, axis=1)
    Wk = _sketch_vectors(u.shape[1], int(ref["sketch_seed"]), int(ref["sketch_k"]), u.device)
    sk = (u @ Wk.T).cpu().numpy()                         # <w_k, u> without conjugation
    e_full = np.sqrt(np.mean(np.abs(sk - ref["sketch"][cols]) ** 2, axis=1)) / ref["norms"][cols]
    norms = torch.linalg.vector_norm(u, dim=1).cpu().numpy()
    e_norm = np.abs(norms - ref["norms"][cols]) / ref["norms"][cols]
    print(f"{label}: max sample rel err {e_samp.max():.2e}, max full-grid (sketch) rel err {e_full.max():.2e}, "
          f"max norm rel diff {e_norm.max():.2e}")
    assert e_samp.max() < tol, (label, e_samp.max())
    assert e_full.max() < tol, (label, e_full.max())
    assert e_norm.max() < tol, (label, e_norm.max())


def test_config3_headline_against_oracle():
    from paper_1801_08655_gb300 import build, hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ref = dict(np.load(GOLDEN))
    p = W.config(3)
    assert np.array_equal(ref["sources"], p.sources)
    assert ref["relres"].max() < 1e-12          # the oracle itself solved the system
    n, N = p.n, p.n ** 3
    rhs = torch.zeros((p.R, n, n, n), dtype=torch.complex128, device="cuda")
    for r, (z, y, x) in enumerate(p.sources):
        rhs[r, z, y, x] = 1.0
    # mixed precision, all 128 right-hand sides, options of the bench
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision="mixed")
    s.factor()
    opts = hz.default_opts("mixed")
    opts.gmres_tol, opts.refine_tol = 1e-4, 1e-5    # the bench's defaults
    u, info, _ = s.solve(rhs, opts)
    s.close()
    del s
    _check(u.reshape(p.R, N), ref, np.arange(p.R), 1e-5, "mixed R=128")
    del u
    torch.cuda.empty_cache()
    # FP64 mode on 8 of the sources (default FP64 options: GMRES to 1e-10)
    cols = np.array([0, 17, 42, 63, 64, 85, 110, 127])
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision="fp64")
    s.factor()
    u, info, _ = s.solve(rhs[torch.from_numpy(cols).cuda()].contiguous())
    s.close()
    _check(u.reshape(len(cols), N), ref, cols, 1e-6, "fp64 R=8")
