"""Write stored oracle values for the 128^3 layered + block workload (all 128 point sources).

Calls only ``oracle/`` (the multifrontal FP64 global direct solve) and the seeded input
generator.  The full solution is 128 x 128^3 complex values (4.3 GB); the fixture keeps, per
right-hand side:
  * a seeded random sample of 512 grid points (``idx``, ``u``),
  * the full-grid and physical-region L2 norms,
  * a sketch: inner products <w_k, u> (no conjugation) with 16 seeded complex Gaussian
    vectors w_k (``numpy.random.default_rng(sketch_seed + k)``, real and imaginary parts
    standard normal divided by sqrt(2)), from which a test estimates the full-grid L2 error
    of another solution without the full reference (E |<w, e>|^2 = ||e||^2),
  * the oracle's own relative residual ||S f - A u|| / ||S f||.

Usage: python tests/golden/make_golden_cfg3.py [spill_dir]
(about 15-30 minutes and 30 GB of memory on 8 cores; the factors, 65 GB, are spilled to
spill_dir, which must have room for them).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import discretization as disc  # noqa: E402
from oracle import multifrontal as mf  # noqa: E402
from paper_1801_08655_gb300 import workloads as W  # noqa: E402

SKETCH_SEED, SKETCH_K, NSAMPLE = 1801128, 16, 512


def sketch_vector(N, k):
    g = np.random.default_rng(SKETCH_SEED + k).standard_normal(2 * N)
    return (g[:N] + 1j * g[N:]) / np.sqrt(2.0)


def main():
    spill = sys.argv[1] if len(sys.argv) > 1 else None
    p = W.config(3)
    n, N = p.n, p.n ** 3
    A = disc.global_operator(p.m, p.omega, p.npml, p.C)
    S = disc.row_scaling(n, p.npml, p.C, p.omega).ravel()
    B = np.zeros((N, p.R), dtype=np.complex128)
    for r, (z, y, x) in enumerate(p.sources):
        c = (z * n + y) * n + x
        B[c, r] = S[c] * 1.0
    t0 = time.time()
    solver = mf.MultifrontalSolver(A, (n, n, n), leaf=512, spill_dir=spill, verbose=True)
    print("symbolic", solver.stats, flush=True)
    X = solver.solve(B)                      # (N, R)
    t1 = time.time()
    res = A @ X - B
    relres = np.linalg.norm(res, axis=0) / np.linalg.norm(B, axis=0)
    del res
    rng = np.random.default_rng(20180125 + 3)
    idx = np.sort(rng.choice(N, size=NSAMPLE, replace=False))
    U = X.T                                   # (R, N) view
    norms = np.linalg.norm(U, axis=1)
    ph = np.zeros((n, n, n), dtype=bool)
    ph[p.npml:n - p.npml, p.npml:n - p.npml, p.npml:n - p.npml] = True
    norms_phys = np.linalg.norm(U[:, ph.ravel()], axis=1)
    sk = np.zeros((p.R, SKETCH_K), dtype=np.complex128)
    for k in range(SKETCH_K):
        sk[:, k] = U @ sketch_vector(N, k)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg3_128cube_layered_block.npz")
    np.savez_compressed(out, idx=idx, u=U[:, idx], norms=norms, norms_phys=norms_phys,
                        sketch=sk, sketch_seed=SKETCH_SEED, sketch_k=SKETCH_K, relres=relres,
                        sources=p.sources, oracle_seconds=t1 - t0)
    print("wrote", out, "oracle solve", round(t1 - t0, 1), "s; max relres", relres.max(), flush=True)


if __name__ == "__main__":
    main()
