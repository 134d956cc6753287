"""Seeded synthetic inputs for the partitioned shift-without-invert eigensolver.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA library (``paper_1606_01139_gb300``).  It synthesises *problem inputs*
only -- grid geometry, the well potential V(r), the two absorbers Gamma_L and
Gamma_R, energy grids and window tables -- and holds none of the method's
arithmetic (no stencil, no Krylov step, no merge, no transmission).

Problem recipe (wire-shaped Kohn-Sham-like operator, Section 1 and Eq. (1)):

* grid: ``nx * ny * nz`` interior points with spacing ``h`` (bohr), flat index
  ``(k * ny + j) * nx + i`` (x fastest).  Coordinates are
  ``x_i = (i - (nx-1)/2) h``, ``y_j = (j - (ny-1)/2) h``, ``z_k = k h``, so the
  wire axis x = y = 0 is the grid's centre line.
* wells: ``V(r) = -sum_w d_w exp(-|r - r_w|^2 / (2 s^2))`` with ``s = 1`` bohr,
  ``r_w = (0, 0, z_w)``, ``z_w ~ U[z_0, z_{nz-1}]`` and ``d_w ~ U[1, 3]`` Ha,
  drawn from ``numpy.random.default_rng(seed)`` (PCG64): first all ``z_w``,
  then all ``d_w``.
* absorbers: planar Gaussians of height 0.5 Ha and standard deviation 2 bohr
  centred on the first and last z planes (the paper's absorbers are Gaussians
  at the two cell ends, Section 1; "width" is read as the standard deviation,
  as the paper states it for its own absorbers in Sections 3.1-3.2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WELL_SIGMA_BOHR = 1.0
ABSORBER_HEIGHT_HA = 0.5
ABSORBER_SIGMA_BOHR = 2.0


@dataclasses.dataclass(frozen=True)
class Wire:
    """A synthetic wire: grid, potential and absorbers (all float64, x fastest)."""

    nx: int
    ny: int
    nz: int
    h: float
    V: np.ndarray
    gamma_L: np.ndarray
    gamma_R: np.ndarray
    z_wells: np.ndarray
    d_wells: np.ndarray

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def coordinates(nx: int, ny: int, nz: int, h: float):
    """Axis coordinates (bohr): x and y centred on the wire axis, z from 0."""
    x = (np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0) * h
    y = (np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0) * h
    z = np.arange(nz, dtype=np.float64) * h
    return x, y, z


def draw_wells(n_wells: int, nz: int, h: float, seed: int):
    """Seeded well positions along the axis and depths (Ha)."""
    rng = np.random.default_rng(seed)
    z_w = rng.uniform(0.0, (nz - 1) * h, size=n_wells)
    d_w = rng.uniform(1.0, 3.0, size=n_wells)
    return z_w, d_w


def well_potential(nx, ny, nz, h, z_w, d_w, sigma=WELL_SIGMA_BOHR):
    """V on the grid as a flat float64 array of length nx*ny*nz (x fastest)."""
    x, y, z = coordinates(nx, ny, nz, h)
    r2_perp = (x[None, :] ** 2 + y[:, None] ** 2)  # [ny, nx]
    V = np.zeros((nz, ny, nx), dtype=np.float64)
    for zw, dw in zip(z_w, d_w):
        dz2 = (z - zw) ** 2  # [nz]
        V -= dw * np.exp(-(dz2[:, None, None] + r2_perp[None, :, :]) / (2.0 * sigma * sigma))
    return V.reshape(-1)


def planar_absorbers(nx, ny, nz, h, height=ABSORBER_HEIGHT_HA, sigma=ABSORBER_SIGMA_BOHR):
    """Gamma_L and Gamma_R: z-Gaussians at the first and last z planes, uniform in x, y."""
    _, _, z = coordinates(nx, ny, nz, h)
    gl = height * np.exp(-((z - z[0]) ** 2) / (2.0 * sigma * sigma))
    gr = height * np.exp(-((z - z[-1]) ** 2) / (2.0 * sigma * sigma))
    ones = np.ones((ny, nx), dtype=np.float64)
    GL = (gl[:, None, None] * ones[None]).reshape(-1)
    GR = (gr[:, None, None] * ones[None]).reshape(-1)
    return GL, GR


def make_wire(nx: int, ny: int, nz: int, h: float = 0.5, n_wells: int = 6, seed: int = 1,
              absorbers: bool = True, wells: bool = True) -> Wire:
    """Build the synthetic wire of the given size (wells and absorbers optional)."""
    z_w, d_w = draw_wells(n_wells, nz, h, seed)
    if wells:
        V = well_potential(nx, ny, nz, h, z_w, d_w)
    else:
        V = np.zeros(nx * ny * nz)
    if absorbers:
        GL, GR = planar_absorbers(nx, ny, nz, h)
    else:
        GL = np.zeros(nx * ny * nz)
        GR = np.zeros(nx * ny * nz)
    return Wire(nx, ny, nz, h, V, GL, GR, z_w, d_w)


def separable_wire(nx: int, ny: int, nz: int, h: float = 0.5, n_wells: int = 6, seed: int = 1,
                   absorbers: bool = True) -> Wire:
    """A wire whose potential depends on z only (wells smeared over x, y).

    ``V(r) = -sum_w d_w exp(-(z - z_w)^2 / 2)``: the operator is then a sum of
    three one-dimensional operators, which gives closed-form spectra at any size.
    """
    z_w, d_w = draw_wells(n_wells, nz, h, seed)
    _, _, z = coordinates(nx, ny, nz, h)
    vz = np.zeros(nz)
    for zw, dw in zip(z_w, d_w):
        vz -= dw * np.exp(-((z - zw) ** 2) / (2.0 * WELL_SIGMA_BOHR ** 2))
    V = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    if absorbers:
        GL, GR = planar_absorbers(nx, ny, nz, h)
    else:
        GL = np.zeros(nx * ny * nz)
        GR = np.zeros(nx * ny * nz)
    return Wire(nx, ny, nz, h, V, GL, GR, z_w, d_w)


# Workloads of the measured configurations (sizes, well counts and seeds).
CONFIGS = {
    # Plain FP64 method, small: 48 lowest pairs in 4 windows, T(E) at 32 energies.
    "wire_10x10x20": dict(nx=10, ny=10, nz=20, h=0.5, n_wells=6, seed=1, n_r=48, p=4,
                          block=8, n_E=32, windows="alg1"),
    # Plain FP64 method, complex128 vectors: 400 pairs in 8 equal-width windows, block 16.
    "wire_48x48x96": dict(nx=48, ny=48, nz=96, h=0.5, n_wells=24, seed=2, n_r=400, p=8,
                          block=16, n_E=128, windows="equal_width"),
    # Mixed-precision form.
    "wire_96x96x192": dict(nx=96, ny=96, nz=192, h=0.5, n_wells=80, seed=3, n_r=2000, p=32,
                           block=16, n_E=0, windows="alg1"),
    # Differentiation form.
    "wire_64x64x128": dict(nx=64, ny=64, nz=128, h=0.5, n_wells=40, seed=5, n_r=1000, p=16,
                           block=16, n_E=256, windows="alg1"),
}


def config_wire(name: str) -> Wire:
    c = CONFIGS[name]
    return make_wire(c["nx"], c["ny"], c["nz"], c["h"], c["n_wells"], c["seed"])


def reduced_wire(name: str, nx: int = 10, ny: int = 10, nz: int = 24) -> Wire:
    """A small copy of a workload for dense-oracle parity: same h, seed and recipe,
    wells scaled with the wire length (n_wells * nz / nz_full, at least 2)."""
    c = CONFIGS[name]
    wells = max(2, int(round(c["n_wells"] * nz / c["nz"])))
    return make_wire(nx, ny, nz, c["h"], wells, c["seed"])


def batch_systems(seed: int = 4, count: int = 64):
    """The uneven batch: per system (nx, ny, nz, n_wells, n_pairs, p, sub_seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        nx = int(rng.integers(16, 49))
        ny = int(rng.integers(16, 49))
        nz = 2 * int(rng.integers(16, 49))
        n_wells = int(rng.integers(8, 41))
        n_pairs = int(rng.integers(32, 257))
        p = int(rng.integers(2, 9))
        out.append(dict(nx=nx, ny=ny, nz=nz, n_wells=n_wells, n_r=n_pairs, p=p, seed=4000 + s))
    return out


def energy_grid(e_lo: float, e_hi: float, n_E: int) -> np.ndarray:
    """``n_E`` uniform energies on [e_lo, e_hi] (Ha)."""
    if n_E == 1:
        return np.array([0.5 * (e_lo + e_hi)])
    return np.linspace(e_lo, e_hi, n_E)


def equal_width_windows(eps_re_sorted: np.ndarray, p: int, inflate: float = 1.1, extra: int = 2):
    """Split [eps_1, eps_n] into p equal-width intervals; shift = interval midpoint.

    Returns (sigma[p], n_req[p]): each request is the interval's count inflated
    by ``inflate`` plus ``extra`` (the paper inflates its requests by 5-10% to
    avoid holes, Section 3).
    """
    lo, hi = float(eps_re_sorted[0]), float(eps_re_sorted[-1])
    edges = np.linspace(lo, hi, p + 1)
    sig = 0.5 * (edges[:-1] + edges[1:])
    counts = np.histogram(eps_re_sorted, bins=edges)[0]
    n_req = np.maximum(1, np.ceil(counts * inflate).astype(int) + extra)
    return sig, n_req


def count_windows(eps_re_sorted: np.ndarray, counts, inflate: float = 1.1, extra: int = 2):
    """Consecutive intervals holding ``counts[j]`` eigenvalues; shift = interval midpoint.

    This is how the paper placed its shifts with foreknowledge of the spectrum
    (Section 3): the sorted spectrum is cut into runs of n_{r,j} values and
    each shift sits at the middle of its run.
    """
    e = np.asarray(eps_re_sorted)
    sig, req = [], []
    start = 0
    for c in counts:
        if start >= len(e):
            break
        stop = min(len(e), start + int(c))
        lo = e[start]
        hi = e[stop - 1]
        sig.append(0.5 * (lo + hi))
        req.append(max(1, int(math.ceil(c * inflate)) + extra))
        start = stop
    return np.array(sig), np.array(req, dtype=int)
