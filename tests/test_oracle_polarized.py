"""Pins of the oracle's step-by-step model of the method (Algorithms 1-9).

Pinned against the global direct solve and against invariants the paper
states: exactness of the Green's representation formula (SIE section,
Theorem 1 of the 2D paper), the sweeps inverting the triangular blocks
(Algorithms 4-5 vs 7-8), the annihilation conditions (Eq. 12) met by the
converged polarized components, the L = 1 and L = 2 special cases, and an
iteration count in the paper's observed range (4-6 per its tables).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import direct, discretization as D, polarized
from paper_1801_08655_gb300 import workloads as W


@pytest.fixture(scope="module")
def case():
    p = W.small_problem(20, 4, 4, seed=31, R=1)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)[0]
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, p.n_layers)
    return p, f[0], u, M


def test_grf_reconstruction_is_exact(case):
    p, f, u, M = case
    t = M.traces_of(u)
    ur = M.reconstruct(f, t)
    assert np.linalg.norm(ur - u) / np.linalg.norm(u) < 1e-13


def test_grf_field_vanishes_on_pad_planes(case):
    p, f, u, M = case
    t = M.traces_of(u)
    for ell in range(M.L):
        g = M.source_part(ell, f)
        if ell >= 1:
            M.S_top(ell, t[ell - 1], g)
        if ell <= M.L - 2:
            M.S_bot(ell, t[ell], g)
        w = M.local_solve(ell, g)
        lo, hi = M.parts[ell]
        zlo, zhi = M.grids[ell]
        pad = np.concatenate([w[:lo - zlo], w[hi - zlo + 1:]])
        assert np.abs(pad).max() <= 1e-13 * np.abs(u).max()


def test_polarized_gmres_matches_direct(case):
    p, f, u, M = case
    us, its = M.solve(f, tol=1e-11)
    assert np.linalg.norm(us - u) / np.linalg.norm(u) < 1e-9
    assert 2 <= its <= 8


def test_sweeps_invert_triangular_blocks(case):
    p, f, u, M = case
    rng = np.random.default_rng(0)
    x = rng.standard_normal(M.zeros_trace().shape) + 1j * rng.standard_normal(M.zeros_trace().shape)
    assert np.abs(M.apply_Dd(M.sweep_down(x)) - x).max() < 1e-12
    assert np.abs(M.apply_Du(M.sweep_up(x)) - x).max() < 1e-12
    # Mpol's diagonal blocks are the same operators
    z = M.zeros_trace()
    dd, du = M.apply_Mpol(x, z)
    assert np.abs(dd - M.apply_Dd(x)).max() < 1e-13
    assert np.abs(du - M.apply_L(x)).max() < 1e-13


def test_annihilation_of_polarized_components(case):
    """Down-going traces generate no field above... in the local operator sense:
    [G^j S_bot u_d_j] on (P_j, Q_j) equals (0, -u_d(Q_j)) (Eq. 12 reading)."""
    p, f, u, M = case
    fd, fu = M.polarized_rhs(f)
    bd, bu = M.apply_P(fd, fu)
    import scipy.sparse.linalg as spla
    b = np.concatenate([bd.ravel(), bu.ravel()])

    def mv(v):
        xd, xu = M._split(v)
        yd, yu = M.apply_P(*M.apply_Mpol(xd, xu))
        return np.concatenate([yd.ravel(), yu.ravel()])

    op = spla.LinearOperator((b.size, b.size), matvec=mv, dtype=complex)
    x, info = spla.gmres(op, b, rtol=1e-12, atol=0, restart=40, maxiter=50)
    ud, uu = M._split(x)
    scale = np.abs(ud).max()
    for j in range(M.K):
        r = M.read_bot(j, M.local_solve(j, M.S_bot(j, ud[j])))
        assert np.abs(r[0]).max() < 1e-8 * scale
        assert np.abs(r[1] + ud[j][1]).max() < 1e-8 * scale
        r = M.read_top(j + 1, M.local_solve(j + 1, M.S_top(j + 1, uu[j])))
        assert np.abs(r[0] + uu[j][0]).max() < 1e-8 * scale
        assert np.abs(r[1]).max() < 1e-8 * scale


def test_single_layer_is_the_global_solve():
    p = W.small_problem(12, 3, 1, seed=41, R=1)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)[0]
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, 1)
    us, its = M.solve(f[0])
    assert its == 0
    assert np.linalg.norm(us - u) / np.linalg.norm(u) < 1e-13


def test_two_layers_diagonal_blocks_are_minus_identity():
    p = W.small_problem(12, 3, 2, seed=43, R=1)
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, 2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(M.zeros_trace().shape) + 0j
    np.testing.assert_array_equal(M.apply_Dd(x), -x)
    np.testing.assert_array_equal(M.apply_Du(x), -x)


def test_exact_green_reductive_case():
    """The reductive case of the Physical intuition subsection: with the local Green's function
    equal to the global one (every layer's local solve replaced by the global direct solve, the
    interface sources and read-outs unchanged), the down-going field has no interface reflections
    (L y_down = 0 to rounding: reflections arise only from truncating the layers) and the
    preconditioned GMRES converges in at most the two iterations the paper states, to the direct
    solution, while the unpreconditioned system needs more.  A dropped identity term in L, for one,
    leaves L y_down at O(1)."""
    n, L = 16, 4
    p = W.small_problem(n, 3, L, seed=5, R=1)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    u = direct.solve(p.m, p.omega, p.npml, p.C, f[None])[0]
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, L)
    G = direct.GlobalSolver(D.global_operator(p.m, p.omega, p.npml, p.C), (n, n, n))
    M.grids = [(0, n - 1)] * L
    M.solvers = [G] * L
    fd, fu = M.polarized_rhs(f)
    yd = M.sweep_down(fd)
    assert np.linalg.norm(M.apply_L(yd)) <= 1e-12 * np.linalg.norm(yd)
    us, its = M.solve(f, tol=1e-12)
    assert its <= 2
    assert np.linalg.norm(us - u) / np.linalg.norm(u) < 1e-12
    M.apply_P = lambda rd, ru: (rd, ru)
    assert M.solve_traces(f, tol=1e-12)[1] > 2


def test_exact_traces_solve_the_sie(case):
    """The SIE reduction (Reduction to a surface integral equation section; Algorithms 2-3): the
    traces of the global solution solve M t = -f_SIE, f_SIE the local fields at the interface
    planes as Algorithm 2 forms them (the sign of reading G2); GMRES on M, matrix-free and
    unpreconditioned, reaches the same traces, and the reconstruction from them is the global
    solution.  The polarized unknowns sum to those traces as well."""
    p, f, u, M = case
    t = M.traces_of(u)
    b = -M.sie_rhs(f)
    r = M.apply_M(t) - b
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
    n = t.size
    op = spla.LinearOperator((n, n), matvec=lambda x: M.apply_M(x.reshape(t.shape)).ravel(), dtype=np.complex128)
    x, info = spla.gmres(op, b.ravel(), rtol=1e-12, atol=0.0, restart=200, maxiter=400)
    assert info == 0
    assert np.linalg.norm(x - t.ravel()) <= 1e-9 * np.linalg.norm(t)
    assert np.linalg.norm(M.reconstruct(f, x.reshape(t.shape)) - u) <= 1e-9 * np.linalg.norm(u)
    ts, _ = M.solve_traces(f, tol=1e-12)
    assert np.linalg.norm(ts - t) <= 1e-9 * np.linalg.norm(t)
