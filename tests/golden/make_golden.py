"""Write stored oracle values for the 64^3 smooth-random workload (16 point sources).

Calls only ``oracle/`` (global FP64 sparse direct solve) and the seeded input generator.
The full solution is 16 x 64^3 complex values; the fixture keeps a seeded random sample
of 4096 grid points per right-hand side plus the 4 interface-adjacent planes' norms,
which the GPU parity test compares against.

Usage: python tests/golden/make_golden.py   (takes a few minutes on one core)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import direct  # noqa: E402
from paper_1801_08655_gb300 import workloads as W  # noqa: E402


def main():
    p = W.config(2)
    f = p.rhs()
    t0 = time.time()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    t1 = time.time()
    rng = np.random.default_rng(20180125)
    n = p.n
    idx = rng.choice(n ** 3, size=4096, replace=False)
    samples = u.reshape(p.R, -1)[:, idx]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_64cube_smooth_samples.npz")
    np.savez_compressed(out, idx=idx, u=samples, norms=np.linalg.norm(u.reshape(p.R, -1), axis=1),
                        oracle_seconds=t1 - t0)
    print("wrote", out, "oracle solve", round(t1 - t0, 1), "s")


if __name__ == "__main__":
    main()
