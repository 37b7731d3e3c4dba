"""Seeded synthetic workloads for the polarized-traces Helmholtz solver.

This module only *generates inputs*: grids, squared-slowness media m(x),
angular frequencies, PML parameters and point-source sets.  It holds none of
the method's arithmetic (no operator, no solve), so that the CPU oracle and
the CUDA path can both draw identical inputs from it without sharing any code
that computes a result.

The media stand in for the paper's test media (homogeneous, smooth random,
"fault"-like layered model; Section "Numerical Experiments"), which the paper
shows only as figures.  Equation convention of the problems generated here:
``Delta u + omega^2 m u = f`` on an n^3 grid with spacing h = 1 (Eq. 1 of the
paper), PML by complex coordinate stretching with the quadratic profile of
the paper's Formulation section.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

__all__ = [
    "Problem",
    "pml_constant",
    "omega_for_ppw",
    "medium_gaussian_bump",
    "medium_smooth_random",
    "medium_layered_block",
    "point_sources_plane_grid",
    "density_smooth_random",
    "config",
    "CONFIG_NAMES",
]


@dataclasses.dataclass
class Problem:
    """One Helmholtz problem: grid, medium, frequency, PML and sources.

    ``m`` is the squared slowness on the full grid (PML included), float64,
    shape (nz, ny, nx) with x fastest.  ``sources`` is an int array of shape
    (R, 3) holding (z, y, x) node indices of unit point sources (value 1/h^3
    with h = 1).
    """

    name: str
    n: int
    npml: int
    n_layers: int
    omega: float
    C: float
    m: np.ndarray
    sources: np.ndarray
    npml_local: int = -1
    h: float = 1.0

    def __post_init__(self):
        if self.npml_local < 0:
            self.npml_local = self.npml

    @property
    def R(self) -> int:
        return int(self.sources.shape[0])

    def rhs(self, dtype=np.complex128) -> np.ndarray:
        """Dense right-hand sides, shape (R, nz, ny, nx), unit point sources."""
        n = self.n
        f = np.zeros((self.R, n, n, n), dtype=dtype)
        for r, (z, y, x) in enumerate(self.sources):
            f[r, z, y, x] = 1.0 / self.h ** 3
        return f


def pml_constant(c_max: float, reflection: float = 1e-3) -> float:
    """PML strength C giving a round-trip normal-incidence reflection ``reflection``.

    With sigma(x) = (C/delta)(x/delta)^2 over a pad of length delta, the
    continuous damping along a round trip is exp(-2 C / (3 c)), so
    C = 1.5 c ln(1/reflection).  The paper leaves C as a tuning parameter
    (Formulation section, after the definition of sigma).
    """
    return 1.5 * c_max * math.log(1.0 / reflection)


def omega_for_ppw(c_min: float, ppw: float, h: float = 1.0) -> float:
    """Angular frequency with ``ppw`` grid points per wavelength at speed c_min."""
    return 2.0 * math.pi * c_min / (ppw * h)


def medium_gaussian_bump(n: int, amp: float = 0.3, width: float = 4.0) -> np.ndarray:
    """c = 1 + amp exp(-|x - x_c|^2 / (2 width^2)) at the grid centre; returns m = 1/c^2."""
    idx = np.arange(n, dtype=np.float64) - (n // 2)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    c = 1.0 + amp * np.exp(-(x * x + y * y + z * z) / (2.0 * width * width))
    return 1.0 / (c * c)


def medium_smooth_random(n: int, seed: int, corr: float = 8.0,
                         cmin: float = 1.5, cmax: float = 4.5) -> np.ndarray:
    """Smooth random medium: white noise, Gaussian low-pass, affine map to [cmin, cmax].

    Noise N(0,1) from ``numpy.random.default_rng(seed)``; the filter kernel is
    exp(-r^2 / corr^2), applied by FFT with periodic wrap; the result is mapped
    affinely so that its min is cmin and its max is cmax.  Returns m = 1/c^2.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n) * n  # integer lags, periodic
    dz, dy, dx = np.meshgrid(k, k, k, indexing="ij")
    ker = np.exp(-(dx * dx + dy * dy + dz * dz) / (corr * corr))
    s = np.real(np.fft.ifftn(np.fft.fftn(w) * np.fft.fftn(ker)))
    s = (s - s.min()) / (s.max() - s.min())
    c = cmin + (cmax - cmin) * s
    return 1.0 / (c * c)


def medium_layered_block(n: int, npml: int, n_vlayers: int = 6,
                         c_top: float = 1.5, c_bot: float = 4.0,
                         c_block: float = 4.5) -> np.ndarray:
    """Flat velocity layers plus a high-velocity block (a stand-in "fault"-like model).

    ``n_vlayers`` equal flat layers over the physical depth with speeds
    linspace(c_top, c_bot); the PML planes above/below take the first/last
    layer's speed.  A block of speed ``c_block`` covers x, y in
    [0.375, 0.625) of the physical extent and velocity layers 2..4 (0-based).
    Returns m = 1/c^2.
    """
    nphys = n - 2 * npml
    speeds = np.linspace(c_top, c_bot, n_vlayers)
    zi = np.arange(n)
    kl = np.clip(((zi - npml) * n_vlayers) // nphys, 0, n_vlayers - 1)
    c = np.empty((n, n, n), dtype=np.float64)
    c[:] = speeds[kl][:, None, None]
    frac = (np.arange(n) - npml) / float(nphys)
    inb = (frac >= 0.375) & (frac < 0.625)
    zsel = (kl >= 2) & (kl <= 4)
    c[np.ix_(zsel, inb, inb)] = c_block
    return 1.0 / (c * c)


def density_smooth_random(n: int, seed: int, corr: float = 6.0, rho_min: float = 1.0,
                          rho_max: float = 2.5) -> np.ndarray:
    """Smooth random mass density: white noise, Gaussian low-pass, affine map to [rho_min, rho_max]
    (the recipe of ``medium_smooth_random``).  Returns b = 1/rho, the coefficient of
    div(b grad u) in the variable-density acoustic operator."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n) * n
    dz, dy, dx = np.meshgrid(k, k, k, indexing="ij")
    ker = np.exp(-(dx * dx + dy * dy + dz * dz) / (corr * corr))
    s = np.real(np.fft.ifftn(np.fft.fftn(w) * np.fft.fftn(ker)))
    s = (s - s.min()) / (s.max() - s.min())
    return 1.0 / (rho_min + (rho_max - rho_min) * s)


def point_sources_plane_grid(n: int, npml: int, z: int, nsx: int, nsy: int) -> np.ndarray:
    """nsx x nsy point sources on plane z, evenly spaced over the physical x, y range."""
    nphys = n - 2 * npml
    xs = [npml + int((ix + 0.5) * nphys / nsx) for ix in range(nsx)]
    ys = [npml + int((iy + 0.5) * nphys / nsy) for iy in range(nsy)]
    out = [(z, y, x) for y in ys for x in xs]
    return np.asarray(out, dtype=np.int64)


CONFIG_NAMES = {
    1: "tiny 24^3 bump, 2 layers, R=1",
    2: "64^3 smooth random, 8 layers, R=16",
    3: "128^3 layered+block, 16 layers, R=128",
    4: "batched uneven: 6 problems 40..96^3",
    5: "serving 160^3 smooth random, 20 layers, 3 frequencies",
}


def _cfg1() -> Problem:
    n, p = 24, 5
    m = medium_gaussian_bump(n)
    src = np.asarray([(n // 2, n // 2, n // 2)], dtype=np.int64)
    return Problem("cfg1_24cube_bump", n, p, 2, omega_for_ppw(1.0, 8.0),
                   pml_constant(1.0), m, src)


def _cfg2() -> Problem:
    n, p = 64, 8
    m = medium_smooth_random(n, seed=1801 + 2)
    src = point_sources_plane_grid(n, p, 10, 4, 4)
    return Problem("cfg2_64cube_smooth", n, p, 8, omega_for_ppw(1.5, 10.0),
                   pml_constant(4.5), m, src)


def _cfg3() -> Problem:
    n, p = 128, 10
    m = medium_layered_block(n, p)
    src = point_sources_plane_grid(n, p, p + 2, 16, 8)
    return Problem("cfg3_128cube_layered_block", n, p, 16, omega_for_ppw(1.5, 8.0),
                   pml_constant(4.5), m, src)


def _cfg4() -> List[Problem]:
    sizes = [40, 48, 64, 64, 80, 96]
    layers = [4, 6, 8, 8, 10, 12]
    rs = [1, 4, 16, 32, 64, 8]
    rng = np.random.default_rng(1801 + 4)
    out = []
    for i, (n, L, R) in enumerate(zip(sizes, layers, rs)):
        p = 8
        m = medium_smooth_random(n, seed=1801 + 40 + i)
        ppw = float(rng.integers(8, 13))
        nphys = n - 2 * p
        sub = rng.choice(nphys * nphys, size=R, replace=False)
        src = np.asarray([(p + 2, p + int(s // nphys), p + int(s % nphys)) for s in sub],
                         dtype=np.int64)
        out.append(Problem(f"cfg4_p{i}_{n}cube", n, p, L, omega_for_ppw(1.5, ppw),
                           pml_constant(4.5), m, src))
    return out


def _cfg5() -> Tuple[np.ndarray, List[float]]:
    n = 160
    m = medium_smooth_random(n, seed=1801 + 5)
    return m, [omega_for_ppw(1.5, ppw) for ppw in (8.0, 10.0, 12.0)]


def config(i: int):
    """Configuration ``i`` (1..5); 4 returns a list of problems, 5 (medium, omegas)."""
    return {1: _cfg1, 2: _cfg2, 3: _cfg3, 4: _cfg4, 5: _cfg5}[i]()


def serving_requests(n: int, npml: int, n_req: int, rate: float, n_omega: int,
                     seed: int = 1801 + 50) -> List[Tuple[float, int, np.ndarray]]:
    """Seeded Poisson request stream: (arrival time [s], omega index, sources (R,3)).

    Each request asks for R ~ U{1..256} point sources drawn without replacement
    from a 16 x 16 grid on plane z = npml + 2.
    """
    rng = np.random.default_rng(seed)
    grid = point_sources_plane_grid(n, npml, npml + 2, 16, 16)
    t = 0.0
    out = []
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate)
        R = int(rng.integers(1, 257))
        sel = np.sort(rng.choice(grid.shape[0], size=R, replace=False))
        out.append((t, int(rng.integers(0, n_omega)), grid[sel]))
    return out


def small_problem(n: int, npml: int, n_layers: int, seed: int = 7, R: int = 2,
                  ppw: float = 8.0, npml_local: int = -1, medium: str = "smooth") -> Problem:
    """A small seeded problem for tests: smooth random (or constant) medium, R sources."""
    if medium == "smooth":
        m = medium_smooth_random(n, seed=seed, corr=max(2.0, n / 8.0))
        cmin, cmax = 1.5, 4.5
    elif medium == "constant":
        m = np.ones((n, n, n))
        cmin = cmax = 1.0
    else:
        raise ValueError(medium)
    rng = np.random.default_rng(seed + 1000)
    nphys = n - 2 * npml
    pts = rng.choice(nphys ** 3, size=R, replace=False)
    src = np.asarray([(npml + int(q // (nphys * nphys)), npml + int((q // nphys) % nphys),
                       npml + int(q % nphys)) for q in pts], dtype=np.int64)
    return Problem(f"small_{n}_{n_layers}_{medium}", n, npml, n_layers,
                   omega_for_ppw(cmin, ppw), pml_constant(cmax), m, src,
                   npml_local=npml_local)
