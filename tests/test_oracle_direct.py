"""Pins of the oracle's global direct solve (the plain definition of the answer).

Dense LAPACK agreement, residual, discrete reciprocity (A is complex
symmetric, so G(x, y) = G(y, x)), and convergence to the analytic free-space
Green's function -exp(i k r) / (4 pi r) of Delta + k^2 in a homogeneous medium
(outgoing convention fixed by Eq. 1 and the sign of i in Eq. 4).
"""
import numpy as np
import pytest

from oracle import direct, discretization as D
from paper_1801_08655_gb300 import workloads as W


def test_nd_order_is_a_permutation():
    for shape in [(5, 6, 7), (17, 24, 24), (1, 3, 9)]:
        p = direct.nd_order(*shape)
        assert np.array_equal(np.sort(p), np.arange(np.prod(shape)))


def test_sparse_matches_dense_lapack():
    p = W.small_problem(10, 3, 1, seed=11, R=3)
    f = p.rhs()
    us = direct.solve(p.m, p.omega, p.npml, p.C, f)
    ud = direct.solve(p.m, p.omega, p.npml, p.C, f, dense=True)
    assert np.linalg.norm(us - ud) / np.linalg.norm(ud) < 1e-12


def test_residual_config1():
    p = W.config(1)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    A = D.global_operator(p.m, p.omega, p.npml, p.C)
    S = D.row_scaling(p.n, p.npml, p.C, p.omega)
    r = A @ u[0].ravel() - (S * f[0]).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(f[0]) <= 1e-12


def test_reciprocity():
    p = W.small_problem(16, 4, 1, seed=21, R=2)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    (z0, y0, x0), (z1, y1, x1) = p.sources
    a, b = u[0, z1, y1, x1], u[1, z0, y0, x0]
    assert abs(a - b) <= 1e-12 * abs(a)


@pytest.mark.slow
def test_free_space_green_function_convergence():
    """Relative L2 error against -exp(ikr)/(4 pi r) over the physical box (r >= 4)
    must be small and fall as the points per wavelength grow; the conjugate
    (incoming) convention must be far off."""
    n, p = 32, 6
    errs = []
    for ppw in (8.0, 12.0):
        m = np.ones((n, n, n))
        om = W.omega_for_ppw(1.0, ppw)
        c = n // 2
        f = np.zeros((1, n, n, n))
        f[0, c, c, c] = 1.0
        u = direct.solve(m, om, p, W.pml_constant(1.0), f)[0]
        idx = np.arange(n) - c
        Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
        r = np.sqrt(X * X + Y * Y + Z * Z)
        mask = np.zeros((n, n, n), bool)
        mask[p:n - p, p:n - p, p:n - p] = True
        mask &= r >= 4
        g = -np.exp(1j * om * r[mask]) / (4 * np.pi * r[mask])
        errs.append(np.linalg.norm(u[mask] - g) / np.linalg.norm(g))
        if ppw == 12.0:
            gc = np.conj(g)
            assert np.linalg.norm(u[mask] - gc) / np.linalg.norm(gc) > 0.5
    assert errs[0] < 0.2 and errs[1] < 0.07
    assert errs[1] < 0.6 * errs[0]
