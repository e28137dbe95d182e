"""Seeded synthetic workloads for the 1D/3D RKETD-FDTD plasma runs.

This module only draws numbers and lays out profiles (cell counts, plasma
frequency and collision-frequency profiles, probe/source cells, frequency
grids). It holds none of the method's arithmetic: no update coefficients,
no field updates, no source pulse and no transforms. Both the CUDA path and
the FP64 oracle receive the arrays built here.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) in counter form, i.e. draw i of a stream
with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15). U(0,1) takes the top 53
bits; N(0,1) uses the Box-Muller transform on consecutive pairs.

Physical setting (paper Sec. IV.B): grid spacing, Courant number 0.5,
Drude plasma slab between vacuum regions, Gaussian-derivative soft source
(Eq. 15) with tau = 15 dt, reflection/transmission probes either side.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+n-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits of each SplitMix64 draw."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on draw pairs (2i, 2i+1)."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1], keeps log finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def dt_for_courant(dz: float, courant: float) -> float:
    """Time step for a Courant number c0*dt/dz."""
    return courant * dz / C0


@dataclass
class Slab1D:
    """One 1D problem: grid, per-cell plasma profile, source and probes (SI)."""

    nz: int
    dz: float
    dt: float
    wp2: np.ndarray  # [nz] plasma frequency squared, rad^2/s^2
    nu: np.ndarray  # [nz] collision frequency, 1/s
    src_cell: int
    src_tau: float
    src_t0: float
    probes: List[int]
    freq_hz: np.ndarray
    bc: str = "mur"  # "mur" or "cpml"
    cpml_cells: int = 0
    steps: int = 0
    src_amp: float = 1.0
    scheme: int = 0  # current recursion: SCHEME_RKETD (Eq. 11), SCHEME_ETD1 (Eq. 9), SCHEME_ETD2 (Eq. 10)

    def vacuum(self) -> "Slab1D":
        """Same grid, source and probes with the plasma removed (incident run)."""
        return Slab1D(self.nz, self.dz, self.dt, np.zeros(self.nz), np.zeros(self.nz), self.src_cell,
                      self.src_tau, self.src_t0, list(self.probes), self.freq_hz, self.bc, self.cpml_cells,
                      self.steps, self.src_amp, self.scheme)


SCHEME_RKETD, SCHEME_ETD1, SCHEME_ETD2 = 0, 1, 2


def c1_plain_slab(nz: int = 2000, steps: int = 8000, slab=(800, 920), wp: float = 2 * math.pi * 28.7e9,
                  nu: float = 2e10, dz: float = 75e-6, courant: float = 0.5) -> Slab1D:
    """Uniform Drude slab of the paper's parameters (Sec. IV.B), scaled to 120 cells (9 mm).

    Source at cell 100, probes at 300 (reflection) and 1700 (transmission), 200 frequencies
    0.5..100 GHz, first-order Mur ends.
    """
    dt = dt_for_courant(dz, courant)
    wp2 = np.zeros(nz)
    nuv = np.zeros(nz)
    wp2[slab[0]:slab[1]] = wp * wp
    nuv[slab[0]:slab[1]] = nu
    tau = 15.0 * dt
    freqs = 0.5e9 * np.arange(1, 201, dtype=np.float64)
    probes = [300, 1700] if nz >= 2000 else [max(2, nz // 8), min(nz - 3, nz - nz // 8)]
    return Slab1D(nz, dz, dt, wp2, nuv, 100 if nz >= 2000 else max(1, nz // 16), tau, 5 * tau, probes,
                  freqs, "mur", 0, steps)


C2_SEED_DENSITY = 0x170900821
C2_SEED_NU = 0x170900822


def c2_epstein(nz: int = 1 << 24, steps: int = 40000, cpml: int = 32, nfreq: int = 512) -> Slab1D:
    """Long inhomogeneous slab: Epstein density ramp with a seeded 5% Gaussian ripple.

    wp2_k = wp0^2 / (1 + exp(-(z_k - z0)/L)) * (1 + 0.05 g_k), clamped at 0, with wp0 = 2pi*50 GHz,
    L = 2 mm, z0 at cell 6032, dz = 1 um; nu_k ~ U[1e9, 5e10]. CPML at both ends, source at
    cell 1032 (tau = 1 ps, t0 = 5 tau), probes at 2032 and 14032, nfreq frequencies to 200 GHz.
    """
    dz = 1e-6
    dt = dt_for_courant(dz, 0.5)
    k = np.arange(nz, dtype=np.float64)
    z = k * dz
    z0 = 6032 * dz
    L = 2e-3
    wp0 = 2 * math.pi * 50e9
    g = normal(C2_SEED_DENSITY, nz)
    with np.errstate(over="ignore"):
        ramp = 1.0 / (1.0 + np.exp(-(z - z0) / L))
    wp2 = np.maximum(wp0 * wp0 * ramp * (1.0 + 0.05 * g), 0.0)
    nu = 1e9 + (5e10 - 1e9) * uniform01(C2_SEED_NU, nz)
    tau = 1e-12
    freqs = 200e9 * np.arange(1, nfreq + 1, dtype=np.float64) / nfreq
    return Slab1D(nz, dz, dt, wp2, nu, 1032, tau, 5 * tau, [2032, 14032], freqs, "cpml", cpml, steps)


C3_SEED = 0x170900823


@dataclass
class Batch1D:
    """A ragged batch of independent 1D slabs sharing dz, dt, source shape and frequencies."""

    slabs: List[Slab1D]
    steps: int

    @property
    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.slabs) + 1, dtype=np.int64)
        off[1:] = np.cumsum([s.nz for s in self.slabs])
        return off

    @property
    def total_cells(self) -> int:
        return int(sum(s.nz for s in self.slabs))


def c3_batch(n_slabs: int = 4096, steps: int = 20000, subset: Optional[List[int]] = None) -> Batch1D:
    """Ragged batch: nz log-uniform in [1024, 65536], slab width 5-40% of nz, uniform plasma.

    Slab i takes draws 4i..4i+3 of stream C3_SEED for (nz, width, wp/2pi in [10, 60] GHz,
    nu in [1e9, 1e11]). dz = 75 um, Courant 0.5, Mur ends, source at 64, probes at 128 and
    256 + width + 64, plasma on [256, 256 + width), tau = 15 dt, 200 frequencies to 100 GHz.
    `subset` selects slab indices (same draws as in the full batch).
    """
    dz = 75e-6
    dt = dt_for_courant(dz, 0.5)
    tau = 15 * dt
    freqs = 0.5e9 * np.arange(1, 201, dtype=np.float64)
    idx = list(range(n_slabs)) if subset is None else list(subset)
    u = uniform01(C3_SEED, 4 * n_slabs)
    slabs = []
    for i in idx:
        u0, u1, u2, u3 = u[4 * i:4 * i + 4]
        nz = int(round(math.exp(math.log(1024) + u0 * (math.log(65536) - math.log(1024)))))
        w = int(math.floor((0.05 + 0.35 * u1) * nz))
        fp = 10e9 + 50e9 * u2
        nu = 1e9 + (1e11 - 1e9) * u3
        wp2 = np.zeros(nz)
        nuv = np.zeros(nz)
        wp2[256:256 + w] = (2 * math.pi * fp) ** 2
        nuv[256:256 + w] = nu
        slabs.append(Slab1D(nz, dz, dt, wp2, nuv, 64, tau, 5 * tau, [128, 256 + w + 64], freqs, "mur", 0, steps))
    return Batch1D(slabs, steps)


C4_SEED_BASE = 0x17090000


def _fourier_profile(seed: int, n: int, modes: int = 16) -> np.ndarray:
    """Smooth random function on [0,1): sum of `modes` Fourier modes with 1/m amplitudes."""
    g = normal(seed, 2 * modes)
    u = (np.arange(n) + 0.5) / n
    s = np.zeros(n)
    for m in range(1, modes + 1):
        s += (g[2 * m - 2] * np.cos(2 * math.pi * m * u) + g[2 * m - 1] * np.sin(2 * math.pi * m * u)) / m
    return s


def c4_profile(i: int, nz: int = 65536, steps: int = 30000, region=(2048, 6144), nfreq: int = 256,
               seed_base: int = C4_SEED_BASE) -> Slab1D:
    """Trainable-profile problem i: smooth random plasma on cells [2048, 6144) of a 65536-cell line.

    wp2 = (2pi*40 GHz)^2 * sigmoid(s(u)) * sin^2(pi u) and nu = 1e9 + 4.9e10 * sigmoid(s'(u)), with
    u the position within the region and s, s' 16-mode Fourier sums from seeds seed_base+i and
    seed_base+i+0x8000. Outside the region wp2 = 0 and nu = nu(s' = 0). Source at 512, reflection
    probe at 1024, Mur ends, tau = 15 dt, nfreq frequencies to 100 GHz.
    """
    dz = 75e-6
    dt = dt_for_courant(dz, 0.5)
    lo, hi = region
    n = hi - lo
    s = _fourier_profile(seed_base + i, n)
    s2 = _fourier_profile(seed_base + i + 0x8000, n)
    u = (np.arange(n) + 0.5) / n
    sig = 1.0 / (1.0 + np.exp(-s))
    sig2 = 1.0 / (1.0 + np.exp(-s2))
    wp2 = np.zeros(nz)
    nu = np.full(nz, 1e9 + 4.9e10 * 0.5)
    wp2[lo:hi] = (2 * math.pi * 40e9) ** 2 * sig * np.sin(math.pi * u) ** 2
    nu[lo:hi] = 1e9 + 4.9e10 * sig2
    tau = 15 * dt
    freqs = 100e9 * np.arange(1, nfreq + 1, dtype=np.float64) / nfreq
    return Slab1D(nz, dz, dt, wp2, nu, 512, tau, 5 * tau, [1024], freqs, "mur", 0, steps)


C4_TARGET_OFFSET = 1000


@dataclass
class Sphere3D:
    """3D problem: cubic grid, plasma sphere, TF/SF plane wave along +z, CPML on all faces."""

    n: int
    d: float
    dt: float
    center: tuple
    radius: float
    wp2: float
    nu: float
    tfsf_lo: int
    tfsf_hi: int
    cpml_cells: int
    src_tau: float
    src_t0: float
    probes: List[tuple]
    freq_hz: np.ndarray
    steps: int


def c5_sphere(n: int = 512, steps: int = 4000, radius: Optional[float] = None, cpml: int = 16,
              nfreq: int = 200) -> Sphere3D:
    """Drude sphere (wp = 2pi*40 GHz, nu = 2e10) in a cubic grid, delta = 100 um, Courant 0.5.

    Radius 120 cells at n = 512 (scaled as n*120/512 otherwise), TF/SF box over cells
    [24*n/512, n - 1 - 24*n/512], Ex-polarised plane wave along +z, probes on the axis
    just outside the TF/SF box on both sides.
    """
    d = 100e-6
    dt = dt_for_courant(d, 0.5)
    r = radius if radius is not None else 120.0 * n / 512.0
    lo = max(cpml + 4, int(round(24 * n / 512)))
    hi = n - 1 - lo
    c = (n // 2, n // 2, n // 2)
    tau = 15 * dt
    freqs = 100e9 * np.arange(1, nfreq + 1, dtype=np.float64) / nfreq
    probes = [(c[0], c[1], lo - 4 if lo - 4 > cpml else lo - 1), (c[0], c[1], hi + 4 if hi + 4 < n - 1 - cpml else hi + 1)]
    return Sphere3D(n, d, dt, c, r, (2 * math.pi * 40e9) ** 2, 2e10, lo, hi, cpml, tau, 5 * tau, probes, freqs, steps)


@dataclass
class Grid3D:
    """A 3D problem on an nx x ny x nz Yee grid (spacing d) with per-cell material indices."""

    nx: int
    ny: int
    nz: int
    d: float
    dt: float
    mat: np.ndarray  # uint8 [nz*ny*nx]: material of Ex, Ey, Ez of the cell in bits 0-1, 2-3, 4-5 (0 = vacuum)
    mat_wp2: np.ndarray  # [n_mat], entry 0 = 0
    mat_nu: np.ndarray
    periodic_xy: bool
    npml: int
    tfsf: bool
    box: tuple  # (i0, i1, j0, j1, k0, k1)
    sheet_k: int
    src_tau: float
    src_t0: float
    probes: List[tuple]
    freq_hz: np.ndarray
    steps: int
    inc_off: int = 8
    inc_len: int = 0
    inc_src: int = 3
    src_amp: float = 1.0

    def __post_init__(self):
        if not self.inc_len:
            self.inc_len = self.nz + 2 * self.inc_off


def sphere_materials(nx: int, ny: int, nz: int, center, radius: float, index: int) -> np.ndarray:
    """Packed per-component material bytes for a sphere: Ex at (i+1/2, j, k), Ey at
    (i, j+1/2, k), Ez at (i, j, k+1/2) take `index` when their own position is inside."""
    k, j, i = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    cx, cy, cz = center
    r2 = radius * radius
    ex = (i + 0.5 - cx) ** 2 + (j - cy) ** 2 + (k - cz) ** 2 <= r2
    ey = (i - cx) ** 2 + (j + 0.5 - cy) ** 2 + (k - cz) ** 2 <= r2
    ez = (i - cx) ** 2 + (j - cy) ** 2 + (k + 0.5 - cz) ** 2 <= r2
    return (ex * index + ey * (index << 2) + ez * (index << 4)).astype(np.uint8).ravel()


def sphere_problem(n: int = 512, steps: int = 4000, radius: Optional[float] = None, npml: int = 16,
                   nfreq: int = 200, box_in: Optional[int] = None) -> Grid3D:
    """Config of the 3D scale-up: Drude sphere (wp = 2pi*40 GHz, nu = 2e10) at the grid centre,
    d = 100 um, Courant 0.5 (c dt/d), CPML on all faces, TF/SF box 24*n/512 cells in from every
    face (box_in cells if given), Ex-polarised plane wave along +z (Eq. 15, tau = 15 dt), probes on
    the axis in the scattered-field region before and after the box."""
    sp = c5_sphere(n=n, steps=steps, radius=radius, cpml=npml, nfreq=nfreq)
    mat = sphere_materials(n, n, n, sp.center, sp.radius, 1)
    lo, hi = sp.tfsf_lo, sp.tfsf_hi
    if box_in is not None:
        lo, hi = box_in, n - 1 - box_in
    return Grid3D(n, n, n, sp.d, sp.dt, mat, np.array([0.0, sp.wp2]), np.array([0.0, sp.nu]), False, npml, True,
                  (lo, hi, lo, hi, lo, hi), -1, sp.src_tau, sp.src_t0, sp.probes, sp.freq_hz, steps)


@dataclass
class Grid2D:
    """A 2D problem (fields uniform along z) on an nx x ny Yee grid of cell size d.

    pol "tm": Ez (i, j), Hx (i, j+1/2), Hy (i+1/2, j); pol "te": Hz (i+1/2, j+1/2), Ex (i+1/2, j),
    Ey (i, j+1/2). Every E component of cell (i, j) takes material mat[j][i] (0 = vacuum). x is
    periodic or bounded by first-order Mur; y by first-order Mur. A soft line source on row src_j
    adds profile[i] s(t) to Ez (tm) or Ex (te); probes (i, j) sample that component."""

    nx: int
    ny: int
    d: float
    dt: float
    pol: str
    periodic_x: bool
    mat: np.ndarray  # uint8 [ny*nx]
    mat_wp2: np.ndarray
    mat_nu: np.ndarray
    src_j: int
    profile: np.ndarray  # [nx]
    src_tau: float
    src_t0: float
    probes: List[tuple]
    freq_hz: np.ndarray
    steps: int
    src_amp: float = 1.0

    def vacuum(self) -> "Grid2D":
        return Grid2D(self.nx, self.ny, self.d, self.dt, self.pol, self.periodic_x, np.zeros_like(self.mat),
                      self.mat_wp2, self.mat_nu, self.src_j, self.profile, self.src_tau, self.src_t0,
                      list(self.probes), self.freq_hz, self.steps, self.src_amp)


def slab_2d(nx: int, ny: int, pol: str, mode: int = 0, d: float = 300e-6, layer=None, wp: float = 2 * math.pi * 28.7e9,
            nu: float = 2e10, steps: int = 8000, periodic_x: bool = True, nfreq: int = 200) -> Grid2D:
    """A plasma layer across a 2D grid (rows layer[0] .. layer[1]-1, default the middle 30 rows), Courant
    0.5 (c dt/d; the 2D limit is 1/sqrt(2)), a line source on row ny/8 with profile cos(2 pi mode i/nx)
    (mode 0: normal incidence; mode m > 0 on a periodic grid: a single transverse Fourier mode, which
    meets the layer at the angle where sin(theta) = m c/(nx d f)), probes on rows ny/4 (reflection) and
    3ny/4 (transmission) in column 0, tau = 15 dt, nfreq frequencies to 100 GHz."""
    dt = dt_for_courant(d, 0.5)
    lo, hi = layer if layer is not None else (ny // 2 - 15, ny // 2 + 15)
    mat = np.zeros((ny, nx), np.uint8)
    mat[lo:hi] = 1
    prof = np.cos(2 * math.pi * mode * np.arange(nx) / nx)
    freqs = 100e9 * np.arange(1, nfreq + 1, dtype=np.float64) / nfreq
    tau = 15 * dt
    return Grid2D(nx, ny, d, dt, pol, periodic_x, mat.ravel(), np.array([0.0, wp * wp]), np.array([0.0, nu]),
                  ny // 8, prof, tau, 5 * tau, [(0, ny // 4), (0, 3 * ny // 4)], freqs, steps)
