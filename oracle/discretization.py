"""Discrete Helmholtz operator with PML (oracle side, FP64, plain numpy/scipy).

Formulation section of the paper: H = Delta_hat + m omega^2 (Eq. 3), with the
stretched derivatives d/dx -> beta_x d/dx, beta_x = 1 / (1 + i sigma_x/omega)
(Eq. 4) and the quadratic profile sigma_x = (C/delta)(x/delta)^2 inside the
absorbing pad, 0 in the physical box (Eq. 5).  Discretized with the standard
second-order 7-point stencil on a regular grid of spacing h.

Reading of the paper where it is silent (the discrete placement of beta):
beta_x d/dx(beta_x d/dx u) is multiplied through by s_x s_y s_z, s = 1/beta =
1 + i sigma/omega, giving the conservative form
    sum_axis d/dx_a ( (s_x s_y s_z / s_a^2) d/dx_a u ) + omega^2 m s_x s_y s_z u,
where the coefficient of axis a is evaluated with s_a at the half node and the
other two factors at the node.  The matrix is then complex symmetric
(A = A^T) and the right-hand side becomes S f, S = s_x s_y s_z (S = 1 in the
physical box).  Dirichlet zero beyond the last grid node.

Sigma origin: the global pad of ``npml`` nodes per face has delta = npml h and
sigma is measured from the first physical node (sigma = 0 at it and inside).
The local pads added at internal layer interfaces start at the half node
beyond the layer's last owned plane, so that the rows of the local operator
on owned planes coincide with the global operator's rows.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "sigma_global",
    "stretch",
    "global_profiles",
    "assemble",
    "global_operator",
    "row_scaling",
    "layer_partition",
    "local_z_sigma",
    "local_operator",
    "local_m",
    "local_b",
    "half_node_average",
]


def sigma_global(x: np.ndarray, n: int, npml: int, C: float, h: float = 1.0) -> np.ndarray:
    """Quadratic PML profile of Eq. 5 at (possibly half-integer) node coordinates x.

    The physical box is nodes [npml, n-1-npml]; the pad length is delta = npml h.
    """
    x = np.asarray(x, dtype=np.float64)
    if npml == 0:
        return np.zeros_like(x)
    delta = npml * h
    lo, hi = float(npml), float(n - 1 - npml)
    d = np.where(x < lo, lo - x, np.where(x > hi, x - hi, 0.0)) * h
    return (C / delta) * (d / delta) ** 2


def stretch(sigma: np.ndarray, omega: float) -> np.ndarray:
    """s = 1/beta = 1 + i sigma/omega (Eq. 4 inverted)."""
    return 1.0 + 1j * np.asarray(sigma, dtype=np.float64) / omega


def global_profiles(n: int, npml: int, C: float, omega: float, h: float = 1.0):
    """(s_node[n], s_half[n+1]) along one axis; s_half[i] sits at coordinate i - 1/2."""
    xn = np.arange(n, dtype=np.float64)
    xh = np.arange(n + 1, dtype=np.float64) - 0.5
    return (stretch(sigma_global(xn, n, npml, C, h), omega),
            stretch(sigma_global(xh, n, npml, C, h), omega))


def half_node_average(b: np.ndarray, axis: int) -> np.ndarray:
    """Values of a nodal field at the half nodes along one axis: entry i sits at i - 1/2 (n + 1
    entries), the average of the two nodes around it; beyond the grid the nearest node stands in."""
    b = np.asarray(b, dtype=np.float64)
    lo = np.take(b, [0], axis=axis)
    hi = np.take(b, [b.shape[axis] - 1], axis=axis)
    ext = np.concatenate([lo, b, hi], axis=axis)
    n = b.shape[axis]
    return 0.5 * (np.take(ext, np.arange(n + 1), axis=axis) + np.take(ext, np.arange(1, n + 2), axis=axis))


def assemble(m: np.ndarray, omega: float, prof_x, prof_y, prof_z, h: float = 1.0,
             b: np.ndarray = None) -> sp.csr_matrix:
    """Assemble the symmetric-form 7-point operator on a box (nz, ny, nx), x fastest.

    prof_a = (s_node[n_a], s_half[n_a + 1]).  Row (k,j,i):
      off-diagonal to (k,j,i+-1):  b(k,j,i+-1/2) s_y(j) s_z(k) / s_x(i +- 1/2) / h^2   (same for y, z)
      diagonal: omega^2 m s_x s_y s_z - (sum of the six couplings, including those
                that reach beyond the grid, whose neighbours are zero).
    b is the nodal coefficient of the divergence-form operator div(b grad u) (b = 1/rho for a
    variable density; None: b = 1, the constant-density Laplacian of Eq. 1), taken at the half
    nodes as the average of its two nodes (half_node_average).
    """
    nz, ny, nx = m.shape
    sxn, sxh = prof_x
    syn, syh = prof_y
    szn, szh = prof_z
    assert sxn.shape == (nx,) and sxh.shape == (nx + 1,)
    assert syn.shape == (ny,) and syh.shape == (ny + 1,)
    assert szn.shape == (nz,) and szh.shape == (nz + 1,)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    gid = (Z * ny + Y) * nx + X
    N = nz * ny * nx
    inv_h2 = 1.0 / (h * h)
    # couplings toward the lower (-) and upper (+) neighbour of every node, per axis
    cxm = syn[Y] * szn[Z] / sxh[X] * inv_h2
    cxp = syn[Y] * szn[Z] / sxh[X + 1] * inv_h2
    cym = sxn[X] * szn[Z] / syh[Y] * inv_h2
    cyp = sxn[X] * szn[Z] / syh[Y + 1] * inv_h2
    czm = sxn[X] * syn[Y] / szh[Z] * inv_h2
    czp = sxn[X] * syn[Y] / szh[Z + 1] * inv_h2
    if b is not None:
        assert b.shape == m.shape
        bx, by, bz = half_node_average(b, 2), half_node_average(b, 1), half_node_average(b, 0)
        cxm, cxp = cxm * bx[Z, Y, X], cxp * bx[Z, Y, X + 1]
        cym, cyp = cym * by[Z, Y, X], cyp * by[Z, Y + 1, X]
        czm, czp = czm * bz[Z, Y, X], czp * bz[Z + 1, Y, X]
    diag = omega ** 2 * m * sxn[X] * syn[Y] * szn[Z] - (cxm + cxp + cym + cyp + czm + czp)
    rows = [gid.ravel()]
    cols = [gid.ravel()]
    vals = [diag.ravel()]

    def add(mask, coef, dz, dy, dx):
        rows.append(gid[mask])
        cols.append(((Z[mask] + dz) * ny + (Y[mask] + dy)) * nx + (X[mask] + dx))
        vals.append(coef[mask])

    add(X > 0, cxm, 0, 0, -1)
    add(X < nx - 1, cxp, 0, 0, 1)
    add(Y > 0, cym, 0, -1, 0)
    add(Y < ny - 1, cyp, 0, 1, 0)
    add(Z > 0, czm, -1, 0, 0)
    add(Z < nz - 1, czp, 1, 0, 0)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N), dtype=np.complex128)
    A.sum_duplicates()
    return A


def global_operator(m: np.ndarray, omega: float, npml: int, C: float, h: float = 1.0,
                    b: np.ndarray = None) -> sp.csr_matrix:
    """Global discrete operator H of Eq. 7 (symmetric form) on the full n^3 grid (b: nodal
    coefficient of div(b grad u), None for the constant-density Laplacian)."""
    n = m.shape[0]
    assert m.shape == (n, n, n)
    p = global_profiles(n, npml, C, omega, h)
    return assemble(m, omega, p, p, p, h, b=b)


def row_scaling(n: int, npml: int, C: float, omega: float, h: float = 1.0) -> np.ndarray:
    """S = s_x s_y s_z on the grid, shape (n, n, n); multiplies f in A u = S f."""
    s, _ = global_profiles(n, npml, C, omega, h)
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


# ----------------------------------------------------------------------------------------------
# layered decomposition (Formulation section, Fig. 1 and Eq. 6)
# ----------------------------------------------------------------------------------------------

def layer_partition(n: int, npml: int, L: int):
    """Owned global plane ranges [(lo, hi)] of the L layers.

    Reading: the physical planes [npml, n-1-npml] are split into L contiguous
    slabs as evenly as possible (earlier layers take the remainder); layer 1
    also owns the top PML planes and layer L the bottom ones.
    """
    nphys = n - 2 * npml
    if L < 1 or nphys < L:
        raise ValueError("need 1 <= L <= number of physical planes")
    q, r = divmod(nphys, L)
    out = []
    start = npml
    for ell in range(L):
        size = q + (1 if ell < r else 0)
        lo, hi = start, start + size - 1
        start += size
        out.append([lo, hi])
    out[0][0] = 0
    out[-1][1] = n - 1
    return [tuple(x) for x in out]


def local_z_sigma(z: np.ndarray, ell: int, parts, n: int, npml: int, npml_local: int, C: float,
                  h: float = 1.0) -> np.ndarray:
    """sigma_z of layer ``ell`` (0-based) at global z coordinates (node or half node).

    Internal interfaces get a fresh pad of npml_local nodes whose profile starts
    at the half node next to the owned planes (mirror above); the global PML is
    inherited at the outer faces.
    """
    z = np.asarray(z, dtype=np.float64)
    L = len(parts)
    lo, hi = parts[ell]
    s = sigma_global(z, n, npml, C, h)
    if npml_local > 0:
        dl = npml_local * h
        if ell > 0:
            top = lo - 0.5
            s = np.where(z < top, (C / dl) * (((top - z) * h) / dl) ** 2, s)
        if ell < L - 1:
            bot = hi + 0.5
            s = np.where(z > bot, (C / dl) * (((z - bot) * h) / dl) ** 2, s)
    return s


def local_grid(ell: int, parts, n: int, npml_local: int):
    """Global z range [zlo, zhi] of layer ell's extended local grid (pads at internal faces)."""
    L = len(parts)
    lo, hi = parts[ell]
    zlo = lo - npml_local if ell > 0 else lo
    zhi = hi + npml_local if ell < L - 1 else hi
    return zlo, zhi


def local_m(m: np.ndarray, ell: int, parts, npml_local: int) -> np.ndarray:
    """m on layer ell's local grid: restriction to the owned planes, extended into
    the pads by copying the nearest owned plane (reading of 'extending m chi')."""
    n = m.shape[0]
    zlo, zhi = local_grid(ell, parts, n, npml_local)
    lo, hi = parts[ell]
    zz = np.clip(np.arange(zlo, zhi + 1), lo, hi)
    return m[zz]


def local_b(b: np.ndarray, ell: int, parts, npml_local: int) -> np.ndarray:
    """b on layer ell's local grid: the owned planes and the one plane beyond each internal
    interface as they are globally (so that the half-node couplings of the owned rows are the
    global ones), copied further into the pads."""
    n = b.shape[0]
    zlo, zhi = local_grid(ell, parts, n, npml_local)
    lo, hi = parts[ell]
    zz = np.clip(np.arange(zlo, zhi + 1), max(lo - 1, 0), min(hi + 1, n - 1))
    return b[zz]


def local_operator(m: np.ndarray, omega: float, ell: int, parts, npml: int, npml_local: int,
                   C: float, h: float = 1.0, b: np.ndarray = None) -> sp.csr_matrix:
    """Local operator H^ell of Eq. 8 on the extended layer (x/y PML inherited)."""
    n = m.shape[0]
    zlo, zhi = local_grid(ell, parts, n, npml_local)
    px = global_profiles(n, npml, C, omega, h)
    zn = np.arange(zlo, zhi + 1, dtype=np.float64)
    zh = np.arange(zlo, zhi + 2, dtype=np.float64) - 0.5
    pz = (stretch(local_z_sigma(zn, ell, parts, n, npml, npml_local, C, h), omega),
          stretch(local_z_sigma(zh, ell, parts, n, npml, npml_local, C, h), omega))
    lb = None if b is None else local_b(b, ell, parts, npml_local)
    return assemble(local_m(m, ell, parts, npml_local), omega, px, px, pz, h, b=lb)
