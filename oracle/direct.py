"""The plain definition of the answer: global FP64 direct solve of A u = S f.

The method of polarized traces converges to exactly the solution of the
global discrete system (the SIE section: the SIE's solution is the
restriction of the global discrete solution to the interfaces, and the
Green's representation formula rebuilds it exactly inside each layer).  So
the oracle for every end-to-end result is this solve, done without any
layering: a dense LAPACK solve on tiny grids, and SuperLU on a
nested-dissection-ordered matrix otherwise.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretization as disc

__all__ = ["nd_order", "GlobalSolver", "solve_dense", "solve"]


def nd_order(nz: int, ny: int, nx: int, leaf: int = 8) -> np.ndarray:
    """Geometric nested-dissection ordering of a box grid (x fastest linear index).

    Recursive bisection of the longest side by a one-node-thick plane; the two
    halves are numbered first, the separator last.  A fill-reducing ordering
    only: it does not change the solution.
    """
    out = []

    def rec(z0, z1, y0, y1, x0, x1):
        dims = (z1 - z0, y1 - y0, x1 - x0)
        if dims[0] <= 0 or dims[1] <= 0 or dims[2] <= 0:
            return
        if dims[0] * dims[1] * dims[2] <= leaf or max(dims) < 3:
            Z, Y, X = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1),
                                  indexing="ij")
            out.append(((Z * ny + Y) * nx + X).ravel())
            return
        a = int(np.argmax(dims))
        if a == 0:
            mid = (z0 + z1) // 2
            rec(z0, mid, y0, y1, x0, x1)
            rec(mid + 1, z1, y0, y1, x0, x1)
            rec(mid, mid + 1, y0, y1, x0, x1)
        elif a == 1:
            mid = (y0 + y1) // 2
            rec(z0, z1, y0, mid, x0, x1)
            rec(z0, z1, mid + 1, y1, x0, x1)
            rec(z0, z1, mid, mid + 1, x0, x1)
        else:
            mid = (x0 + x1) // 2
            rec(z0, z1, y0, y1, x0, mid)
            rec(z0, z1, y0, y1, mid + 1, x1)
            rec(z0, z1, y0, y1, mid, mid + 1)

    rec(0, nz, 0, ny, 0, nx)
    perm = np.concatenate(out)
    assert perm.size == nz * ny * nx
    return perm


class GlobalSolver:
    """Sparse direct factorization of a box operator, reusable for many RHS.

    A is permuted by ``nd_order`` and handed to SuperLU with the natural
    column order; threshold partial pivoting is kept (diag_pivot_thresh 0.1)
    so the oracle does not depend on the no-pivot stability the GPU path
    relies on.
    """

    def __init__(self, A: sp.spmatrix, shape):
        nz, ny, nx = shape
        self.perm = nd_order(nz, ny, nx)
        self.iperm = np.empty_like(self.perm)
        self.iperm[self.perm] = np.arange(self.perm.size)
        Ap = sp.csc_matrix(A)[self.perm][:, self.perm]
        self.lu = spla.splu(sp.csc_matrix(Ap), permc_spec="NATURAL", diag_pivot_thresh=0.1,
                            options=dict(SymmetricMode=True))

    def solve(self, b: np.ndarray) -> np.ndarray:
        """Solve for b of shape (N,) or (N, k)."""
        bp = b[self.perm]
        xp = self.lu.solve(np.ascontiguousarray(bp))
        return xp[self.iperm]


def solve_dense(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """Dense LAPACK (partially pivoted LU) solve; tiny grids only."""
    return sla.solve(A.toarray(), b)


def solve(m: np.ndarray, omega: float, npml: int, C: float, f: np.ndarray,
          h: float = 1.0, dense: bool = False, b: np.ndarray = None) -> np.ndarray:
    """u solving A u = S f for f of shape (R, n, n, n); returns u of the same shape (b: nodal
    coefficient of div(b grad u), None for constant density)."""
    n = m.shape[0]
    A = disc.global_operator(m, omega, npml, C, h, b=b)
    S = disc.row_scaling(n, npml, C, omega, h)
    B = (S[None] * f).reshape(f.shape[0], -1).T
    if dense:
        X = solve_dense(A, B)
    else:
        X = GlobalSolver(A, (n, n, n)).solve(B)
    return X.T.reshape(f.shape)
