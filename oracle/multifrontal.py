"""Multifrontal FP64 direct solve of A u = b on a box grid -- TEST INFRASTRUCTURE ONLY.

The third tier of the oracle, for grids where SuperLU's single thread and memory do not
reach (96^3 - 160^3).  It computes the same thing as ``direct.solve``: the global discrete
solution of A u = S f (the SIE section: the method converges to exactly that solution), only
organised as the paper organises its own local solves ("Local Solves: Parallel Multi-frontal
Methods" section: a fill-reducing nested-dissection reordering, then a multifrontal
factorization and forward/backward substitution).  Written to be read against the textbook
definition of block Gaussian elimination, not for speed:

* ordering: recursive bisection of the box by one-node-thick planes (``dissection_tree``);
  every tree node owns its separator (or leaf box), children before parents;
* symbolic phase, generic (no geometric shortcut): the update set of a node is the set of
  later-eliminated unknowns coupled to its own unknowns, either directly in A or through a
  child's update set (``symbolic``); that every such unknown is eliminated later is checked,
  which is the condition that the tree is an assembly tree of A;
* numeric phase, children before parents: the front F = [F11 F12; F21 F22] over (own, update)
  is assembled from A's entries in the own rows and columns plus the children's update
  matrices (extend-add); F11 is factored by LAPACK LU with partial pivoting (the oracle does
  not rely on the unpivoted stability the GPU path uses); the update matrix for the parent is
  the Schur complement F22 - F21 F11^{-1} F12;
* the forward substitution runs inside the factorization (y1 = F11^{-1} b1, b2 -= F21 y1);
  the backward substitution runs parents before children (x1 = y1 - F11^{-1} F12 x2) and
  needs only (LU(F11), F12) per node, which can be spilled to disk for the largest grids.

Threads: the dense LAPACK/BLAS calls use the BLAS library's threads; the tree is walked in
order by one Python thread.
"""
from __future__ import annotations

import dataclasses
import os
import shutil
import tempfile
import time
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import discretization as disc

__all__ = ["TreeNode", "dissection_tree", "symbolic", "MultifrontalSolver", "solve"]


@dataclasses.dataclass
class TreeNode:
    own: np.ndarray                 # natural cell ids owned by the node (its separator or leaf box)
    children: List[int]
    s: int = 0                      # own unknowns are elimination indices [s, t)
    t: int = 0
    upd: Optional[np.ndarray] = None  # sorted elimination indices of the update set


def dissection_tree(nz: int, ny: int, nx: int, leaf: int = 512) -> List[TreeNode]:
    """Nested-dissection tree of an (nz, ny, nx) box grid, nodes in post-order (children first).

    A box of more than ``leaf`` cells (and a side of at least 3) is cut across its longest
    side by the one-cell plane through its middle; the two halves become the children and the
    plane is the node's own set.  Smaller boxes are leaves owning all their cells.
    """
    nodes: List[TreeNode] = []

    def cells(z0, z1, y0, y1, x0, x1):
        Z, Y, X = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        return ((Z * ny + Y) * nx + X).ravel()

    def build(box) -> int:
        z0, z1, y0, y1, x0, x1 = box
        dims = (z1 - z0, y1 - y0, x1 - x0)
        if dims[0] * dims[1] * dims[2] <= leaf or max(dims) < 3:
            nodes.append(TreeNode(own=cells(*box), children=[]))
            return len(nodes) - 1
        a = int(np.argmax(dims))
        lo, hi = box[2 * a], box[2 * a + 1]
        mid = (lo + hi) // 2
        b1, b2, sep = list(box), list(box), list(box)
        b1[2 * a + 1] = mid
        b2[2 * a] = mid + 1
        sep[2 * a], sep[2 * a + 1] = mid, mid + 1
        kids = [build(tuple(b1)), build(tuple(b2))]
        nodes.append(TreeNode(own=cells(*sep), children=kids))
        return len(nodes) - 1

    build((0, nz, 0, ny, 0, nx))
    e = 0
    for nd in nodes:
        nd.s, nd.t = e, e + nd.own.size
        e = nd.t
    assert e == nz * ny * nx
    return nodes


def symbolic(nodes: List[TreeNode], Ap: sp.csr_matrix) -> None:
    """Update sets of every node from the graph of the permuted matrix Ap (elimination order).

    upd(k) = ( {j : Ap[i, j] != 0, i own by k} U  union of upd(c) over children c ) minus
    own(k).  The tree is an assembly tree of A only if every coupling of k's own unknowns to an
    earlier-eliminated unknown stays inside k's subtree (post-order makes the subtree the index
    range [first_k, t_k)) and no child's update set reaches an unknown eliminated before k;
    both are checked, since the elimination below would be wrong otherwise.
    """
    first = []
    for nd in nodes:
        f = min([first[c] for c in nd.children], default=nd.s)
        first.append(f)
        cols = Ap.indices[Ap.indptr[nd.s]:Ap.indptr[nd.t]]
        if np.any(cols < f):
            raise ValueError("dissection tree is not an assembly tree of A (coupling leaves the subtree)")
        parts = [cols[cols >= nd.t]]
        for c in nd.children:
            u = nodes[c].upd
            if np.any(u < nd.s):
                raise ValueError("dissection tree is not an assembly tree of A (update set reaches a sibling)")
            parts.append(u[u >= nd.t])
        nd.upd = np.unique(np.concatenate(parts))


class MultifrontalSolver:
    """Multifrontal factorization of a sparse box operator with its right-hand sides.

    ``solve(B)`` factors A and runs both substitutions for the columns of B (N x R, natural
    order) in one pass; the factors are not kept afterwards (one call per operator).
    """

    def __init__(self, A: sp.spmatrix, shape, leaf: int = 512, spill_dir: Optional[str] = None,
                 spill_min_entries: int = 1 << 22, verbose: bool = False):
        nz, ny, nx = shape
        self.nodes = dissection_tree(nz, ny, nx, leaf)
        self.perm = np.concatenate([nd.own for nd in self.nodes])          # elimination -> cell
        self.iperm = np.empty_like(self.perm)
        self.iperm[self.perm] = np.arange(self.perm.size)
        A = sp.csr_matrix(A)
        self.Ap = sp.csr_matrix(A[self.perm][:, self.perm])                # rows and columns permuted
        self.Ap.sort_indices()
        self.Apc = sp.csc_matrix(self.Ap)
        self.Apc.sort_indices()
        symbolic(self.nodes, self.Ap)
        self.spill_dir = spill_dir
        self.spill_min = spill_min_entries
        self.verbose = verbose
        self.stats = dict(nodes=len(self.nodes), max_front=max(nd.own.size + nd.upd.size for nd in self.nodes),
                          factor_entries=int(sum(nd.own.size * (nd.own.size + nd.upd.size) for nd in self.nodes)))

    # ------------------------------------------------------------------ one front
    def _assemble(self, nd: TreeNode, loc: np.ndarray, updates) -> np.ndarray:
        no, nu = nd.t - nd.s, nd.upd.size
        m = no + nu
        F = np.zeros((m, m), dtype=np.complex128, order="F")
        # original entries in the own columns (all rows of the front) ...
        sl = slice(self.Apc.indptr[nd.s], self.Apc.indptr[nd.t])
        rows = self.Apc.indices[sl]
        cnt = np.diff(self.Apc.indptr[nd.s:nd.t + 1])
        colj = np.repeat(np.arange(no), cnt)
        keep = rows >= nd.s
        r = loc[rows[keep]]
        assert np.all(r >= 0), "a coupled unknown is missing from the front"
        F[r, colj[keep]] = self.Apc.data[sl][keep]
        # ... and in the own rows, update columns (the own x own block is already in place)
        sl = slice(self.Ap.indptr[nd.s], self.Ap.indptr[nd.t])
        cols = self.Ap.indices[sl]
        cnt = np.diff(self.Ap.indptr[nd.s:nd.t + 1])
        rowi = np.repeat(np.arange(no), cnt)
        keep = cols >= nd.t
        c = loc[cols[keep]]
        assert np.all(c >= 0), "a coupled unknown is missing from the front"
        F[rowi[keep], c] = self.Ap.data[sl][keep]
        # extend-add of the children's update matrices
        for c in nd.children:
            U = updates.pop(c)
            p = loc[self.nodes[c].upd]
            F[np.ix_(p, p)] += U
            del U
        return F

    def solve(self, B: np.ndarray) -> np.ndarray:
        """Solve A X = B for B of shape (N,) or (N, R) in natural order."""
        vec = B.ndim == 1
        Y = np.array(B[self.perm].reshape(self.perm.size, -1), dtype=np.complex128, order="C")
        N = self.perm.size
        loc = np.full(N, -1, dtype=np.int64)
        updates = {}
        stored = []
        tmp = None
        if self.spill_dir is not None:
            os.makedirs(self.spill_dir, exist_ok=True)
            tmp = tempfile.mkdtemp(prefix="mf_", dir=self.spill_dir)
        t0 = time.time()
        try:
            # ---- factorization with the forward substitution, children before parents
            for k, nd in enumerate(self.nodes):
                no = nd.t - nd.s
                idx = np.concatenate([np.arange(nd.s, nd.t), nd.upd])
                loc[idx] = np.arange(idx.size)
                F = self._assemble(nd, loc, updates)
                loc[idx] = -1
                lu = sla.lu_factor(F[:no, :no], check_finite=False)            # F11 = P L U
                F12 = np.asfortranarray(F[:no, no:])
                F21 = F[no:, :no]
                y1 = sla.lu_solve(lu, Y[nd.s:nd.t], check_finite=False)         # y1 = F11^{-1} b1
                Y[nd.s:nd.t] = y1
                if nd.upd.size:
                    Y[nd.upd] -= F21 @ y1                                        # b2 -= F21 y1
                    X = sla.lu_solve(lu, F12, check_finite=False)                # F11^{-1} F12
                    U = np.asfortranarray(F[no:, no:])
                    U -= F21 @ X                                                 # Schur complement
                    updates[k] = U
                    del X
                del F, F21
                item = (lu[0], lu[1], F12)
                if tmp is not None and lu[0].size + F12.size >= self.spill_min:
                    path = os.path.join(tmp, f"n{k}.npz")
                    np.savez(path, lu=lu[0], piv=lu[1], f12=F12)
                    item = path
                stored.append(item)
                if self.verbose and no + nd.upd.size > 4000:
                    print(f"  node {k}/{len(self.nodes)} front {no}+{nd.upd.size} "
                          f"t={time.time() - t0:.0f}s", flush=True)
            assert not updates
            # ---- backward substitution, parents before children
            for k in range(len(self.nodes) - 1, -1, -1):
                nd = self.nodes[k]
                item = stored[k]
                if isinstance(item, str):
                    with np.load(item) as z:
                        item = (z["lu"], z["piv"], z["f12"])
                    os.remove(stored[k])
                lu0, piv, F12 = item
                if nd.upd.size:
                    Y[nd.s:nd.t] -= sla.lu_solve((lu0, piv), F12 @ Y[nd.upd], check_finite=False)
                stored[k] = None
        finally:
            if tmp is not None:
                shutil.rmtree(tmp, ignore_errors=True)
        X = Y[self.iperm]
        return X[:, 0] if vec else X


def solve(m: np.ndarray, omega: float, npml: int, C: float, f: np.ndarray, h: float = 1.0,
          leaf: int = 512, spill_dir: Optional[str] = None, verbose: bool = False) -> np.ndarray:
    """u solving A u = S f for f of shape (R, n, n, n) by the multifrontal method."""
    n = m.shape[0]
    A = disc.global_operator(m, omega, npml, C, h)
    S = disc.row_scaling(n, npml, C, omega, h)
    B = (S[None] * f).reshape(f.shape[0], -1).T
    X = MultifrontalSolver(A, (n, n, n), leaf=leaf, spill_dir=spill_dir, verbose=verbose).solve(B)
    return X.T.reshape(f.shape)
