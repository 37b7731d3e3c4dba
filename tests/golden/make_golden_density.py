"""Write stored oracle values for the variable-density workload: the 64^3 smooth-random medium of
the 64^3 workload (8 layers, 16 point sources on z = 10) with a seeded smooth random density
rho in [1, 2.5] (b = 1/rho, workloads.density_smooth_random(64, 1801 + 22)).

Calls only ``oracle/`` (global FP64 sparse direct solve of div(b grad u) + omega^2 m u = S f) and
the seeded input generators.  Keeps 4096 seeded sample points per right-hand side and the full
norms, like the constant-density fixture.

Usage: python tests/golden/make_golden_density.py   (a few minutes on one core)
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
    b = W.density_smooth_random(p.n, seed=1801 + 22)
    f = p.rhs()
    t0 = time.time()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f, b=b)
    t1 = time.time()
    rng = np.random.default_rng(20180125 + 22)
    idx = rng.choice(p.n ** 3, size=4096, replace=False)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_64cube_density_samples.npz")
    np.savez_compressed(out, idx=idx, u=u.reshape(p.R, -1)[:, idx], norms=np.linalg.norm(u.reshape(p.R, -1), axis=1),
                        density_seed=1801 + 22, oracle_seconds=t1 - t0)
    print("wrote", out, "oracle solve", round(t1 - t0, 1), "s")


if __name__ == "__main__":
    main()
