"""Step-by-step CPU model of the method of polarized traces (oracle side, FP64).

Follows the paper in its own order: Algorithm 1 (factor each layer's local
operator), Algorithm 2 (partition the source, local solves, form the trace
right-hand side, solve the trace system, reconstruct each layer with the
Green's representation formula), the polarized system of Eq. 13-14 with the
Gauss-Seidel preconditioner of Eq. 16, the sweeps of Algorithms 4-5, the
reflections of Algorithm 6 and the matrix-free blocks of Algorithms 7-9 in
the appendix.  Local solves use SciPy's SuperLU; GMRES is SciPy's.

Indices are 0-based here: layers ell = 0..L-1, interfaces j = 0..K-1 with
K = L-1; interface j separates layers j and j+1 and carries the plane pair
(P_j, Q_j) = (last owned plane of layer j, first owned plane of layer j+1).
A trace pair is stored as an array (2, ny, nx) = (t(P_j), t(Q_j)); a trace
vector is (K, 2, ny, nx).  In the paper's local numbering, planes n, n+1 of
layer ell are (P_ell, Q_ell) and planes 0, 1 are (P_{ell-1}, Q_{ell-1}).

Readings where the printed algorithms are garbled (each checked by the pins
in tests/test_oracle_polarized.py against the global direct solve):
* Dirac-delta sources (delta(z - z_p) v / h^3 in the Formulation section):
  the interface source weights are taken from the assembled matrix itself, so
  that they match the discrete Green's representation formula exactly:
  S_top(t_{j}) for layer j+1 puts -c t(P_j) on plane Q_j and +c t(Q_j) on the
  pad plane P_j; S_bot(t_j) for layer j puts -c t(Q_j) on plane P_j and
  +c t(P_j) on the pad plane Q_j, with c = A[(z,y,x),(z+-1,y,x)] = s_x s_y / h^2
  at a physical half plane.
* Algorithm 6, layer L uses the down-going input (the printed up-arrow on the
  source line contradicts the two lines after it).
* Algorithm 8 is the application of D-up, not its inverse (its body uses the
  input v throughout, mirroring Algorithm 7).
* Algorithm 9 (U) is the mirror image of Algorithm 6: for layer ell, the
  local field due to both of its interfaces' up-going traces, read on its
  bottom pair, minus the input on plane P.
* Explicit trace-to-trace blocks (trace_blocks): the paper applies the blocks of its trace
  operators only matrix-free (never forming the SIE matrix in 3D); written out, a block is the
  local Green's function between two interface pairs, R_rd G^ell R_src^T J_src, with J_src the
  interface source's weights, which makes E_rs J_s^{-1} = (E_sr J_r^{-1})^T by the complex
  symmetry of the local operator (pinned).
* The polarized right-hand side, which the paper obtains from the SIE right-hand side by
  rearrangements it does not print (Polarization subsection): f_down_j = -(v^j(P_j), v^j(Q_j)),
  f_up_j = -(v^{j+1}(P_j), v^{j+1}(Q_j)), with v^ell the local solution for the
  layer's own part of the source (Algorithm 2, local solves).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import discretization as disc
from .direct import GlobalSolver

__all__ = ["PolarizedModel"]


class PolarizedModel:
    """Algorithm 1 at construction; the online blocks as methods."""

    def __init__(self, m, omega, npml, C, L, npml_local=None, h=1.0, b=None):
        self.m = np.asarray(m, dtype=np.float64)
        self.n = n = self.m.shape[0]
        self.omega, self.npml, self.C, self.L, self.h = omega, npml, C, L, h
        self.npml_local = npml if npml_local is None else npml_local
        self.parts = disc.layer_partition(n, npml, L)
        self.K = L - 1
        self.b = None if b is None else np.asarray(b, dtype=np.float64)
        s, _ = disc.global_profiles(n, npml, C, omega, h)
        self.c0 = (s[None, :] * s[:, None]) / (h * h)  # s_y(y) s_x(x) / h^2
        self.S = disc.row_scaling(n, npml, C, omega, h)
        self.grids = []
        self.solvers = []
        # Algorithm 1: build and factor every local operator
        for ell in range(L):
            zlo, zhi = disc.local_grid(ell, self.parts, n, self.npml_local)
            H = disc.local_operator(self.m, omega, ell, self.parts, npml, self.npml_local, C, h, b=self.b)
            self.grids.append((zlo, zhi))
            self.solvers.append(GlobalSolver(H, (zhi - zlo + 1, n, n)))

    # ------------------------------------------------------------------ local primitives
    def nz_local(self, ell):
        zlo, zhi = self.grids[ell]
        return zhi - zlo + 1

    def zeros_local(self, ell):
        return np.zeros((self.nz_local(ell), self.n, self.n), dtype=np.complex128)

    def local_solve(self, ell, g):
        """w = (H^ell)^{-1} g on the local grid (g shape (nz_loc, n, n))."""
        w = self.solvers[ell].solve(g.reshape(-1))
        return w.reshape(g.shape)

    def plane(self, ell, w, z):
        """Value of a local field w of layer ell on global plane z."""
        return w[z - self.grids[ell][0]]

    def add_plane(self, ell, g, z, v):
        g[z - self.grids[ell][0]] += v

    def coupling(self, P):
        """c = A[(Q,y,x),(P,y,x)] across the physical half plane between planes P and Q = P+1:
        s_y s_x / h^2, times b at that half plane for a variable density."""
        if self.b is None:
            return self.c0
        return self.c0 * 0.5 * (self.b[P] + self.b[P + 1])

    def S_top(self, ell, pair, g=None):
        """Interface source of interface ell-1 acting on layer ell (ell >= 1)."""
        g = self.zeros_local(ell) if g is None else g
        P = self.parts[ell - 1][1]
        Q = P + 1
        c = self.coupling(P)
        self.add_plane(ell, g, Q, -c * pair[0])
        self.add_plane(ell, g, P, c * pair[1])
        return g

    def S_bot(self, ell, pair, g=None):
        """Interface source of interface ell acting on layer ell (ell <= L-2)."""
        g = self.zeros_local(ell) if g is None else g
        P = self.parts[ell][1]
        Q = P + 1
        c = self.coupling(P)
        self.add_plane(ell, g, P, -c * pair[1])
        self.add_plane(ell, g, Q, c * pair[0])
        return g

    def read_bot(self, ell, w):
        """Paper's planes (n, n+1) of layer ell = (P_ell, Q_ell)."""
        P = self.parts[ell][1]
        return np.stack([self.plane(ell, w, P), self.plane(ell, w, P + 1)])

    def read_top(self, ell, w):
        """Paper's planes (0, 1) of layer ell = (P_{ell-1}, Q_{ell-1})."""
        Q = self.parts[ell][0]
        return np.stack([self.plane(ell, w, Q - 1), self.plane(ell, w, Q)])

    def zeros_trace(self):
        return np.zeros((self.K, 2, self.n, self.n), dtype=np.complex128)

    # ------------------------------------------------------------------ Algorithm 2 pieces
    def source_part(self, ell, f):
        """f^ell = f chi_{Omega^ell}, scaled by S, on layer ell's local grid."""
        g = self.zeros_local(ell)
        lo, hi = self.parts[ell]
        zlo = self.grids[ell][0]
        g[lo - zlo:hi - zlo + 1] = (self.S * f)[lo:hi + 1]
        return g

    def local_fields(self, f):
        """v^ell = (H^ell)^{-1} f^ell for every layer (Algorithm 2, local solves)."""
        return [self.local_solve(ell, self.source_part(ell, f)) for ell in range(self.L)]

    def polarized_rhs(self, f):
        v = self.local_fields(f)
        fd, fu = self.zeros_trace(), self.zeros_trace()
        for j in range(self.K):
            fd[j] = -self.read_bot(j, v[j])
            fu[j] = -self.read_top(j + 1, v[j + 1])
        return fd, fu

    def reconstruct(self, f, t):
        """Local reconstruction with interface sources (Algorithm 2, inner solves)."""
        u = np.zeros((self.n,) * 3, dtype=np.complex128)
        for ell in range(self.L):
            g = self.source_part(ell, f)
            if ell >= 1:
                self.S_top(ell, t[ell - 1], g)
            if ell <= self.L - 2:
                self.S_bot(ell, t[ell], g)
            w = self.local_solve(ell, g)
            lo, hi = self.parts[ell]
            zlo = self.grids[ell][0]
            u[lo:hi + 1] = w[lo - zlo:hi - zlo + 1]
        return u

    # ------------------------------------------------------------------ SIE matrix (Algorithm 3)
    def sie_rhs(self, f):
        """Right-hand side of the SIE as Algorithm 2 forms it: for interface j, the local fields of
        the two layers at the interface's planes, (v^j(P_j), v^{j+1}(Q_j))."""
        v = self.local_fields(f)
        out = self.zeros_trace()
        for j in range(self.K):
            P = self.parts[j][1]
            out[j] = np.stack([self.plane(j, v[j], P), self.plane(j + 1, v[j + 1], P + 1)])
        return out

    def apply_M(self, t):
        """Application of the SIE matrix (Algorithm 3), matrix-free: every layer's local solve with
        the interface sources of the traces on both of its interfaces, read on the layer's own
        boundary planes, minus the input there: (M t)_j = (w^j(P_j) - t_j(P), w^{j+1}(Q_j) - t_j(Q)).
        Read as G1 (the layer-2 source of the first step is v^2_1, the first output is u^1 at plane
        n^1).  With the interface weights of the assembled matrix (R7) the exact traces solve
        M t = -sie_rhs(f): the Green's representation formula gives t = v + w(t) on those planes."""
        K, L = self.K, self.L
        out = self.zeros_trace()
        w = []
        for ell in range(L):
            g = self.zeros_local(ell)
            if ell >= 1:
                self.S_top(ell, t[ell - 1], g)
            if ell <= L - 2:
                self.S_bot(ell, t[ell], g)
            w.append(self.local_solve(ell, g))
        for j in range(K):
            P = self.parts[j][1]
            out[j] = np.stack([self.plane(j, w[j], P) - t[j][0], self.plane(j + 1, w[j + 1], P + 1) - t[j][1]])
        return out

    # ------------------------------------------------------------------ blocks of M_pol
    def apply_Mpol(self, xd, xu):
        """Application of the polarized matrix (appendix): u_d = D_d x_d + U x_u,
        u_u = D_u x_u + L x_d (Algorithms 7, 9, 8, 6)."""
        K, L = self.K, self.L
        wA = [None] * L
        wB = [None] * L
        wC = [None] * L
        wD = [None] * L
        for ell in range(L):
            if ell >= 1:
                wA[ell] = self.local_solve(ell, self.S_top(ell, xd[ell - 1]))
                wC[ell] = self.local_solve(ell, self.S_top(ell, xu[ell - 1]))
            if ell <= L - 2:
                wB[ell] = self.local_solve(ell, self.S_bot(ell, xd[ell]))
                wD[ell] = self.local_solve(ell, self.S_bot(ell, xu[ell]))
        Dd, U, Du, Lx = (self.zeros_trace() for _ in range(4))
        for j in range(K):
            # Algorithm 7: D_down
            Dd[j] = -xd[j] if j == 0 else self.read_bot(j, wA[j]) - xd[j]
            # Algorithm 9 (read as the mirror of Algorithm 6): U
            w = wD[j] if j == 0 else wD[j] + wC[j]
            r = self.read_bot(j, w)
            U[j] = np.stack([r[0] - xu[j][0], r[1]])
            # Algorithm 8: D_up
            Du[j] = -xu[j] if j == K - 1 else self.read_top(j + 1, wD[j + 1]) - xu[j]
            # Algorithm 6: L
            w = wA[j + 1] if j + 1 == L - 1 else wA[j + 1] + wB[j + 1]
            r = self.read_top(j + 1, w)
            Lx[j] = np.stack([r[0], r[1] - xd[j][1]])
        return Dd + U, Du + Lx

    def apply_L(self, xd):
        """Algorithm 6 alone (upward reflections)."""
        out = self.zeros_trace()
        for j in range(self.K):
            ell = j + 1
            g = self.S_top(ell, xd[j])
            if ell <= self.L - 2:
                self.S_bot(ell, xd[ell], g)
            r = self.read_top(ell, self.local_solve(ell, g))
            out[j] = np.stack([r[0], r[1] - xd[j][1]])
        return out

    def apply_Dd(self, xd):
        out = self.zeros_trace()
        for j in range(self.K):
            out[j] = -xd[j] if j == 0 else \
                self.read_bot(j, self.local_solve(j, self.S_top(j, xd[j - 1]))) - xd[j]
        return out

    def apply_Du(self, xu):
        out = self.zeros_trace()
        for j in range(self.K):
            out[j] = -xu[j] if j == self.K - 1 else \
                self.read_top(j + 1, self.local_solve(j + 1, self.S_bot(j + 1, xu[j + 1]))) - xu[j]
        return out

    def sweep_down(self, r):
        """Algorithm 4: (D_down)^{-1} r by a sequential downward sweep."""
        y = self.zeros_trace()
        y[0] = -r[0]
        for j in range(1, self.K):
            y[j] = self.read_bot(j, self.local_solve(j, self.S_top(j, y[j - 1]))) - r[j]
        return y

    def sweep_up(self, s):
        """Algorithm 5: (D_up)^{-1} s by a sequential upward sweep."""
        y = self.zeros_trace()
        y[-1] = -s[-1]
        for j in range(self.K - 2, -1, -1):
            y[j] = self.read_top(j + 1, self.local_solve(j + 1, self.S_bot(j + 1, y[j + 1]))) - s[j]
        return y

    def apply_P(self, rd, ru):
        """Gauss-Seidel preconditioner of Eq. 16: [[D_d, 0], [L, D_u]]^{-1}."""
        yd = self.sweep_down(rd)
        yu = self.sweep_up(ru - self.apply_L(yd))
        return yd, yu

    # ------------------------------------------------------------------ explicit trace blocks
    def trace_blocks(self):
        """Explicit trace-to-trace Green's blocks of every layer: the local Green's function
        between the layer's interface plane pairs, i.e. the blocks that Algorithms 4-9 apply
        matrix-free by local solves with interface sources, written out as dense matrices.

        Returns a list over layers of dicts: E[ell][rd + src] with rd, src in {'t', 'b'} is the
        dense (2P x 2P) matrix taking a trace pair on the layer's top interface (src 't', interface
        ell-1, through S_top) or bottom interface (src 'b', interface ell, through S_bot) to the
        layer's top (rd 't': planes P_{ell-1}, Q_{ell-1}) or bottom (rd 'b': P_ell, Q_ell) read-out
        pair.  Pairs are flattened as (plane, y, x).  Column k is the local solution for the k-th
        unit trace, so a block is one local solve with 2P right-hand sides."""
        n, L = self.n, self.L
        p2 = 2 * n * n
        unit = np.eye(p2, dtype=np.complex128).reshape(p2, 2, n, n)
        out = []
        for ell in range(L):
            blocks = {}
            for src in ("t", "b"):
                if (src == "t" and ell == 0) or (src == "b" and ell == L - 1):
                    continue
                inject = self.S_top if src == "t" else self.S_bot
                G = np.stack([inject(ell, e).ravel() for e in unit], axis=1)
                W = self.solvers[ell].solve(G).T.reshape(p2, self.nz_local(ell), n, n)
                if ell >= 1:
                    blocks["t" + src] = np.stack([self.read_top(ell, w).ravel() for w in W], axis=1)
                if ell <= L - 2:
                    blocks["b" + src] = np.stack([self.read_bot(ell, w).ravel() for w in W], axis=1)
            out.append(blocks)
        return out

    def _blk(self, B, v):
        return (B @ v.ravel()).reshape(2, self.n, self.n)

    def apply_Mpol_blocks(self, E, xd, xu):
        """M_pol from the explicit blocks: the local solves of Algorithms 6-9 replaced by block
        products.  Down rows: -x_d - [plane P] x_u + E_bt (x_d + x_u) of the interface above +
        E_bb x_u; up rows: -x_u - [plane Q] x_d + E_tt x_d + E_tb (x_d + x_u) of the interface
        below (blocks of layer j for down row j, of layer j+1 for up row j)."""
        K, L = self.K, self.L
        ud, uu = -xd.copy(), -xu.copy()
        ud[:, 0] -= xu[:, 0]
        uu[:, 1] -= xd[:, 1]
        for j in range(K):
            if j >= 1:
                ud[j] += self._blk(E[j]["bt"], xd[j - 1] + xu[j - 1])
            ud[j] += self._blk(E[j]["bb"], xu[j])
            uu[j] += self._blk(E[j + 1]["tt"], xd[j])
            if j + 1 <= L - 2:
                uu[j] += self._blk(E[j + 1]["tb"], xd[j + 1] + xu[j + 1])
        return ud, uu

    def apply_P_blocks(self, E, rd, ru):
        """The preconditioner of Eq. 16 from the explicit blocks: downward sweep (Algorithm 4)
        y_d_j = E^j_bt y_d_{j-1} - r_d_j; reflections (Algorithm 6) s = r_u - L y_d; upward
        sweep (Algorithm 5) y_u_j = E^{j+1}_tb y_u_{j+1} - s_j."""
        K, L = self.K, self.L
        yd, yu = self.zeros_trace(), self.zeros_trace()
        yd[0] = -rd[0]
        for j in range(1, K):
            yd[j] = self._blk(E[j]["bt"], yd[j - 1]) - rd[j]
        s = ru.copy()
        s[:, 1] += yd[:, 1]
        for j in range(K):
            s[j] -= self._blk(E[j + 1]["tt"], yd[j])
            if j + 1 <= L - 2:
                s[j] -= self._blk(E[j + 1]["tb"], yd[j + 1])
        yu[K - 1] = -s[K - 1]
        for j in range(K - 2, -1, -1):
            yu[j] = self._blk(E[j + 1]["tb"], yu[j + 1]) - s[j]
        return yd, yu

    # ------------------------------------------------------------------ GMRES (Eq. 15)
    def _split(self, v):
        k = self.K * 2 * self.n * self.n
        return v[:k].reshape(self.K, 2, self.n, self.n), v[k:].reshape(self.K, 2, self.n, self.n)

    def solve_traces(self, f, tol=1e-10, restart=40, maxiter=200, blocks=None):
        """Left-preconditioned GMRES on P M_pol u = P f_pol, x0 = 0; returns (t, iterations).
        With `blocks` (from trace_blocks) M_pol and P are applied by explicit block products."""
        if self.L == 1:
            return self.zeros_trace(), 0
        if blocks is None:
            Pc, Mp = self.apply_P, self.apply_Mpol
        else:
            Pc = lambda a, b: self.apply_P_blocks(blocks, a, b)       # noqa: E731
            Mp = lambda a, b: self.apply_Mpol_blocks(blocks, a, b)    # noqa: E731
        fd, fu = self.polarized_rhs(f)
        bd, bu = Pc(fd, fu)
        b = np.concatenate([bd.ravel(), bu.ravel()])

        def mv(v):
            xd, xu = self._split(v)
            yd, yu = Pc(*Mp(xd, xu))
            return np.concatenate([yd.ravel(), yu.ravel()])

        op = spla.LinearOperator((b.size, b.size), matvec=mv, dtype=np.complex128)
        its = [0]

        def cb(_):
            its[0] += 1

        x, info = spla.gmres(op, b, rtol=tol, atol=0.0, restart=restart, maxiter=maxiter,
                             callback=cb, callback_type="pr_norm")
        xd, xu = self._split(x)
        return xd + xu, its[0]

    def solve(self, f, tol=1e-10, blocks=None):
        """Full online solve (Algorithm 2) for one right-hand side f (n, n, n)."""
        t, its = self.solve_traces(f, tol, blocks=blocks)
        return self.reconstruct(f, t), its

    def traces_of(self, u):
        """Restriction of a global field u to the interface plane pairs."""
        t = self.zeros_trace()
        for j in range(self.K):
            P = self.parts[j][1]
            t[j] = np.stack([u[P], u[P + 1]])
        return t
