"""Pins of the oracle's operator assembly (Formulation section, Eqs. 3-7).

Each check is independent of the assembly code it tests: Kronecker sums of
1D stretched second differences, the textbook 7-point Laplacian, closed-form
values of the quadratic PML profile, and exact complex symmetry.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretization as D
from paper_1801_08655_gb300 import workloads as W


def _kron_operator(m, omega, npml, C):
    """Separable construction: sum over axes of (diag of the other two s) x (1D
    operator d/dx (1/s) d/dx), plus omega^2 m s_x s_y s_z on the diagonal."""
    n = m.shape[0]
    x = np.arange(n, dtype=float)
    sig_n = np.zeros(n)
    sig_h = np.zeros(n + 1)
    if npml > 0:
        lo, hi, dl = npml, n - 1 - npml, float(npml)
        for i in range(n):
            d = max(lo - x[i], x[i] - hi, 0.0)
            sig_n[i] = C / dl * (d / dl) ** 2
        for i in range(n + 1):
            xh = i - 0.5
            d = max(lo - xh, xh - hi, 0.0)
            sig_h[i] = C / dl * (d / dl) ** 2
    sn = 1 + 1j * sig_n / omega
    sh = 1 + 1j * sig_h / omega
    inv = 1.0 / sh
    D1 = sp.diags([-(inv[:-1] + inv[1:]), inv[1:-1], inv[1:-1]], [0, -1, 1], shape=(n, n))
    Sd = sp.diags(sn)
    I = sp.identity(n)
    # linear index (z, y, x) with x fastest => kron(z, y, x)
    A = (sp.kron(Sd, sp.kron(Sd, D1)) + sp.kron(Sd, sp.kron(D1, Sd)) + sp.kron(D1, sp.kron(Sd, Sd)))
    S = np.einsum("i,j,k->ijk", sn, sn, sn).ravel()
    A = A + sp.diags(omega ** 2 * m.ravel() * S)
    return sp.csr_matrix(A), S


@pytest.mark.parametrize("npml", [0, 3])
def test_assembly_matches_kronecker_construction(npml):
    n = 11
    p = W.small_problem(n, max(npml, 1), 1, seed=3, R=1)
    m = p.m
    A = D.global_operator(m, p.omega, npml, p.C)
    B, S = _kron_operator(m, p.omega, npml, p.C)
    assert abs(A - B).max() < 1e-12 * abs(B).max()
    np.testing.assert_allclose(D.row_scaling(n, npml, p.C, p.omega).ravel(), S, rtol=1e-14, atol=0)


def test_no_pml_is_textbook_seven_point_laplacian():
    n = 7
    m = np.full((n, n, n), 0.25)
    omega = 1.3
    A = D.global_operator(m, omega, 0, 10.0).toarray()
    N = n ** 3
    ref = np.zeros((N, N))
    for z in range(n):
        for y in range(n):
            for x in range(n):
                g = (z * n + y) * n + x
                ref[g, g] = -6.0 + omega ** 2 * 0.25
                for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < n and 0 <= yy < n and 0 <= xx < n:
                        ref[g, (zz * n + yy) * n + xx] = 1.0
    np.testing.assert_array_equal(A, ref.astype(complex))


def test_pml_profile_closed_form():
    n, p, C = 20, 5, 7.0
    s = D.sigma_global(np.arange(n, dtype=float), n, p, C)
    # first physical node and everything inside: zero
    assert np.all(s[p:n - p] == 0.0)
    # outermost node: distance delta -> sigma = C/delta
    assert s[0] == pytest.approx(C / p)
    assert s[n - 1] == pytest.approx(C / p)
    # half way into the pad: (C/delta) (1/2)^2
    sh = D.sigma_global(np.array([p - p / 2.0]), n, p, C)
    assert sh[0] == pytest.approx(C / p * 0.25)
    # symmetric in the two faces
    np.testing.assert_allclose(s, s[::-1])


def test_operator_is_complex_symmetric_and_not_hermitian():
    p = W.config(1)
    A = D.global_operator(p.m, p.omega, p.npml, p.C)
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 0.1


def test_layer_partition_even_split_and_pml_ownership():
    parts = D.layer_partition(128, 10, 16)
    assert parts[0][0] == 0 and parts[-1][1] == 127
    sizes = [hi - lo + 1 for lo, hi in parts]
    phys = [s for s in sizes]
    phys[0] -= 10
    phys[-1] -= 10
    assert sum(phys) == 108 and max(phys) - min(phys) <= 1
    for (a, b), (c, d) in zip(parts[:-1], parts[1:]):
        assert c == b + 1


def test_local_operator_rows_on_owned_planes_equal_global_rows():
    """The local pads start half a cell past the owned planes, so H^ell agrees
    with H on every owned row (needed for the exact Green's representation)."""
    p = W.small_problem(16, 3, 3, seed=5, R=1)
    n = p.n
    A = D.global_operator(p.m, p.omega, p.npml, p.C).tocsr()
    parts = D.layer_partition(n, p.npml, 3)
    for ell in range(3):
        H = D.local_operator(p.m, p.omega, ell, parts, p.npml, p.npml, p.C).tocsr()
        zlo, zhi = D.local_grid(ell, parts, n, p.npml)
        lo, hi = parts[ell]
        for z in (lo, (lo + hi) // 2, hi):
            for (y, x) in [(0, 0), (5, 7), (n - 1, n - 1)]:
                g = (z * n + y) * n + x
                gl = ((z - zlo) * n + y) * n + x
                rg = A.getrow(g).toarray().ravel()
                rl = H.getrow(gl).toarray().ravel()
                # map local columns to global ones
                cols = np.nonzero(rl)[0]
                zc = cols // (n * n) + zlo
                gc = zc * n * n + cols % (n * n)
                assert np.allclose(rg[gc], rl[cols], rtol=0, atol=1e-14)
                assert np.count_nonzero(rg) == cols.size
