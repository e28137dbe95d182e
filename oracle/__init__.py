"""FP64 CPU oracle for the RKETD-FDTD scheme -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this package. The product path (the CUDA library and its Python
binding) never imports it. The C sources here are compiled with gcc into
oracle/_build/ (serial build and an OpenMP build of the same file).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["rketd_oracle.c", "rketd_oracle3d.c", "rketd_oracle2d.c"]
_LOCK = threading.Lock()
_LIBS = {}


def build(omp: bool = False, force: bool = False, mutant: int = 0) -> str:
    """Compiles the oracle with gcc (-O2 -ffp-contract=off); returns the .so path.

    `mutant` > 0 builds a copy with one planted mistake (tests only: they check
    that the pins reject it).
    """
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle_omp.so" if omp else "liboracle.so"
    if mutant:
        name = f"liboracle_mut{mutant}.so"
    out = os.path.join(_BUILD, name)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    if omp:
        cmd.append("-fopenmp")
    if mutant:
        cmd.append(f"-DOR_MUTANT={int(mutant)}")
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(cmd + srcs + ["-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


class OrGrid1D(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int64), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc", ctypes.c_int32), ("cpml_cells", ctypes.c_int32),
        ("cpml_m", ctypes.c_double), ("cpml_sigma_max", ctypes.c_double),
        ("cpml_kappa_max", ctypes.c_double), ("cpml_alpha_max", ctypes.c_double),
        ("src_cell", ctypes.c_int64), ("src_tau", ctypes.c_double), ("src_t0", ctypes.c_double),
        ("src_amp", ctypes.c_double), ("n_probes", ctypes.c_int32), ("n_freq", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
    ]


class OrGrid3D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("d", ctypes.c_double),
                ("dt", ctypes.c_double), ("periodic_xy", ctypes.c_int32), ("npml", ctypes.c_int32),
                ("pml_m", ctypes.c_double), ("pml_sigma_max", ctypes.c_double), ("pml_kappa_max", ctypes.c_double),
                ("pml_alpha_max", ctypes.c_double), ("tfsf", ctypes.c_int32), ("box", ctypes.c_int32 * 6),
                ("sheet_k", ctypes.c_int32), ("src_tau", ctypes.c_double), ("src_t0", ctypes.c_double),
                ("src_amp", ctypes.c_double), ("n_probes", ctypes.c_int32), ("n_freq", ctypes.c_int32),
                ("inc_off", ctypes.c_int32), ("inc_len", ctypes.c_int32), ("inc_src", ctypes.c_int32)]


class OrGrid2D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("d", ctypes.c_double), ("dt", ctypes.c_double),
                ("pol", ctypes.c_int32), ("periodic_x", ctypes.c_int32), ("src_j", ctypes.c_int32),
                ("src_tau", ctypes.c_double), ("src_t0", ctypes.c_double), ("src_amp", ctypes.c_double),
                ("n_probes", ctypes.c_int32), ("n_freq", ctypes.c_int32)]


def lib(omp: bool = False, mutant: int = 0) -> ctypes.CDLL:
    key = (omp, mutant)
    with _LOCK:
        if key not in _LIBS:
            L = ctypes.CDLL(build(omp, mutant=mutant))
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int64)
            L.or_run1d.argtypes = [ctypes.POINTER(OrGrid1D), dp, dp, ip, dp, ctypes.c_int64, ctypes.c_int64,
                                   dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.or_run1d.restype = ctypes.c_int
            L.or_phi1.argtypes = [ctypes.c_double]
            L.or_phi1.restype = ctypes.c_double
            L.or_phi2.argtypes = [ctypes.c_double]
            L.or_phi2.restype = ctypes.c_double
            L.or_threads.restype = ctypes.c_int
            L.or_dphi1.argtypes = [ctypes.c_double]
            L.or_dphi1.restype = ctypes.c_double
            L.or_dphi2.argtypes = [ctypes.c_double]
            L.or_dphi2.restype = ctypes.c_double
            L.or_adjoint_step.argtypes = [ctypes.POINTER(OrGrid1D), dp, dp, dp, dp, dp]
            L.or_adjoint_step.restype = ctypes.c_int
            L.or_adjoint1d.argtypes = [ctypes.POINTER(OrGrid1D), dp, dp, ip, dp, ctypes.c_int64, dp, dp, dp, dp]
            L.or_adjoint1d.restype = ctypes.c_int
            L.or_run3d.argtypes = [ctypes.POINTER(OrGrid3D), ctypes.POINTER(ctypes.c_uint8), dp, dp, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32), dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                   dp, dp, dp]
            L.or_run3d.restype = ctypes.c_int
            L.or_run2d.argtypes = [ctypes.POINTER(OrGrid2D), ctypes.POINTER(ctypes.c_uint8), dp, dp, ctypes.c_int32,
                                   dp, ctypes.POINTER(ctypes.c_int32), dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                   dp]
            L.or_run2d.restype = ctypes.c_int
            _LIBS[key] = L
        return _LIBS[key]


def cpml_defaults(dz: float, m: float = 3.0):
    """CPML grading used for the long-domain runs: m = 3, sigma_max = 0.8 (m+1)/(eta0 dz),
    kappa_max = 1, alpha_max = 0.05 S/m."""
    eta0 = np.sqrt(1.25663706212e-6 / 8.8541878128e-12)
    return m, 0.8 * (m + 1) / (eta0 * dz), 1.0, 0.05


def make_grid(slab, cpml=None) -> OrGrid1D:
    g = OrGrid1D()
    g.nz = slab.nz
    g.dz = slab.dz
    g.dt = slab.dt
    g.bc = {"mur": 0, "cpml": 1, "pml": 2}[slab.bc]
    g.cpml_cells = slab.cpml_cells if slab.bc in ("cpml", "pml") else 0
    m, smax, kmax, amax = cpml if cpml is not None else cpml_defaults(slab.dz)
    g.cpml_m, g.cpml_sigma_max, g.cpml_kappa_max, g.cpml_alpha_max = m, smax, kmax, amax
    g.src_cell = slab.src_cell
    g.src_tau = slab.src_tau
    g.src_t0 = slab.src_t0
    g.src_amp = slab.src_amp
    g.n_probes = len(slab.probes)
    g.n_freq = len(slab.freq_hz)
    g.scheme = slab.scheme
    return g


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class State1D:
    """Oracle state in SI units: E^n, H^{n-1/2}, J^n, CPML memories, DFT sums, step index."""

    def __init__(self, slab):
        nz = slab.nz
        self.E = np.zeros(nz)
        self.H = np.zeros(nz - 1)
        self.J = np.zeros(nz)
        self.psiE = np.zeros(nz)
        self.psiH = np.zeros(nz - 1)
        self.X = np.zeros((len(slab.probes), len(slab.freq_hz)), dtype=np.complex128)
        self.Eprev = np.zeros(nz)  # E^{n-1}, carried by the explicit second-order scheme (Eq. 10)
        self.n = 0

    def copy(self):
        c = object.__new__(State1D)
        for k, v in self.__dict__.items():
            setattr(c, k, v.copy() if isinstance(v, np.ndarray) else v)
        return c


def run1d(slab, steps: Optional[int] = None, state: Optional[State1D] = None, series: bool = False,
          omp: bool = False, cpml=None, mutant: int = 0):
    """Runs the oracle for `steps` steps (default slab.steps) from `state` (default zero fields).

    Returns (state, series) where series is [n_probes, steps] or None.
    """
    L = lib(omp, mutant)
    steps = slab.steps if steps is None else steps
    st = State1D(slab) if state is None else state
    g = make_grid(slab, cpml)
    wp2 = np.ascontiguousarray(slab.wp2, dtype=np.float64)
    nu = np.ascontiguousarray(slab.nu, dtype=np.float64)
    probes = np.ascontiguousarray(np.asarray(slab.probes, dtype=np.int64))
    freqs = np.ascontiguousarray(slab.freq_hz, dtype=np.float64)
    xr = np.ascontiguousarray(st.X.real.copy())
    xi = np.ascontiguousarray(st.X.imag.copy())
    ser = np.zeros((len(slab.probes), steps)) if series else None
    rc = L.or_run1d(ctypes.byref(g), _dp(wp2), _dp(nu), probes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    _dp(freqs), st.n, steps, _dp(st.E), _dp(st.H), _dp(st.J), _dp(st.psiE), _dp(st.psiH),
                    _dp(xr), _dp(xi), _dp(ser) if ser is not None else ctypes.POINTER(ctypes.c_double)(),
                    _dp(st.Eprev))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    st.X = xr + 1j * xi
    st.n += steps
    return st, ser


def phi1(x: float) -> float:
    return lib().or_phi1(x)


def phi2(x: float) -> float:
    return lib().or_phi2(x)


def threads(omp: bool = True) -> int:
    return lib(omp).or_threads()


def reflection_transmission(X_tot: np.ndarray, X_inc: np.ndarray):
    """R = (X_R^tot - X_R^inc)/X_R^inc at probe 0 and T = X_T^tot/X_T^inc at probe 1."""
    R = (X_tot[0] - X_inc[0]) / X_inc[0]
    T = X_tot[1] / X_inc[1] if X_tot.shape[0] > 1 else None
    return R, T


def dphi1(x: float) -> float:
    return lib().or_dphi1(x)


def dphi2(x: float) -> float:
    return lib().or_dphi2(x)


def adjoint_step(slab, lE, lH, lJ):
    """One transposed step (Mur ends, no gradients): returns the adjoint before the step."""
    g = make_grid(slab)
    lE = np.ascontiguousarray(lE, float).copy()
    lH = np.ascontiguousarray(np.concatenate([lH, [0.0]]), float)
    lJ = np.ascontiguousarray(lJ, float).copy()
    rc = lib().or_adjoint_step(ctypes.byref(g), _dp(np.ascontiguousarray(slab.wp2, float)),
                               _dp(np.ascontiguousarray(slab.nu, float)), _dp(lE), _dp(lH), _dp(lJ))
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return lE, lH[:-1], lJ


def adjoint(slab, gX: np.ndarray, steps: Optional[int] = None):
    """dL/d(wp2), dL/d(nu) per cell for a loss with dL/dX = gX ([n_probes, n_freq] complex:
    real part dL/dRe X, imaginary part dL/dIm X) after `steps` steps from rest."""
    g = make_grid(slab)
    steps = slab.steps if steps is None else steps
    gr = np.ascontiguousarray(np.real(gX).ravel(), float)
    gi = np.ascontiguousarray(np.imag(gX).ravel(), float)
    gw = np.zeros(slab.nz)
    gn = np.zeros(slab.nz)
    probes = np.ascontiguousarray(np.asarray(slab.probes, dtype=np.int64))
    rc = lib().or_adjoint1d(ctypes.byref(g), _dp(np.ascontiguousarray(slab.wp2, float)),
                            _dp(np.ascontiguousarray(slab.nu, float)),
                            probes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _dp(np.ascontiguousarray(slab.freq_hz, float)), steps, _dp(gr), _dp(gi), _dp(gw), _dp(gn))
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return gw, gn


def reflection_loss(X_tot, X_inc, R_target):
    """L = sum_f (|R(f)| - |R_t(f)|)^2 with R = (X_R^tot - X_R^inc)/X_R^inc at probe 0, and
    dL/dX (complex: dL/dRe X + j dL/dIm X) for every probe (zero except probe 0)."""
    d = X_tot[0] - X_inc[0]
    absr = np.abs(d) / np.abs(X_inc[0])
    L = float(np.sum((absr - R_target) ** 2))
    # d|d|/dRe d = Re d/|d|, d|d|/dIm d = Im d/|d|
    coef = 2.0 * (absr - R_target) / (np.abs(X_inc[0]) * np.abs(d))
    gX = np.zeros_like(X_tot)
    gX[0] = coef * d.real + 1j * coef * d.imag
    return L, gX


class State3D:
    """3D oracle state: fields [9][N] (Ex, Ey, Ez, Hx, Hy, Hz, Jx, Jy, Jz), CPML memories
    [12][N], incident line [2][L], DFT sums, step index."""

    def __init__(self, prob):
        N = prob.nx * prob.ny * prob.nz
        self.fields = np.zeros((9, N))
        self.psi = np.zeros((12, N))
        self.inc = np.zeros((2, prob.inc_len))
        self.X = np.zeros((len(prob.probes), len(prob.freq_hz)), dtype=np.complex128)
        self.n = 0

    def field(self, name, prob):
        i = ["Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Jx", "Jy", "Jz"].index(name)
        return self.fields[i].reshape(prob.nz, prob.ny, prob.nx)


def run3d(prob, steps=None, state=None, series=False, mutant: int = 0):
    """Runs the 3D oracle on a workloads.Grid3D problem (`mutant` > 0: a build with one planted
    mistake, for the tests that check the pins reject it)."""
    L = lib(mutant=mutant)
    steps = prob.steps if steps is None else steps
    st = State3D(prob) if state is None else state
    g = OrGrid3D()
    g.nx, g.ny, g.nz, g.d, g.dt = prob.nx, prob.ny, prob.nz, prob.d, prob.dt
    g.periodic_xy = 1 if prob.periodic_xy else 0
    g.npml = prob.npml
    g.pml_m, g.pml_sigma_max, g.pml_kappa_max, g.pml_alpha_max = cpml_defaults(prob.d)
    g.tfsf = 1 if prob.tfsf else 0
    for q in range(6):
        g.box[q] = prob.box[q]
    g.sheet_k = prob.sheet_k
    g.src_tau, g.src_t0, g.src_amp = prob.src_tau, prob.src_t0, prob.src_amp
    g.n_probes, g.n_freq = len(prob.probes), len(prob.freq_hz)
    g.inc_off, g.inc_len, g.inc_src = prob.inc_off, prob.inc_len, prob.inc_src
    mat = np.ascontiguousarray(prob.mat, dtype=np.uint8)
    mw = np.ascontiguousarray(prob.mat_wp2, float)
    mn = np.ascontiguousarray(prob.mat_nu, float)
    pr = np.ascontiguousarray(np.asarray(prob.probes, np.int32).ravel())
    fr = np.ascontiguousarray(prob.freq_hz, float)
    xr = np.ascontiguousarray(st.X.real.copy())
    xi = np.ascontiguousarray(st.X.imag.copy())
    ser = np.zeros((len(prob.probes), steps)) if series else None
    rc = L.or_run3d(ctypes.byref(g), mat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dp(mw), _dp(mn), len(mw),
                    pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(fr), st.n, steps, _dp(st.fields),
                    _dp(st.psi), _dp(st.inc), _dp(xr), _dp(xi),
                    _dp(ser) if ser is not None else ctypes.POINTER(ctypes.c_double)())
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    st.X = xr + 1j * xi
    st.n += steps
    return st, ser


FIELDS_2D = {"tm": ("Ez", "Hx", "Hy", "Jz"), "te": ("Ex", "Ey", "Hz", "Jx", "Jy")}


class State2D:
    """2D oracle state: fields [6][ny*nx] (TMz: Ez, Hx, Hy, Jz; TEz: Ex, Ey, Hz, Jx, Jy), DFT sums, step."""

    def __init__(self, prob):
        self.fields = np.zeros((6, prob.nx * prob.ny))
        self.X = np.zeros((len(prob.probes), len(prob.freq_hz)), dtype=np.complex128)
        self.n = 0

    def field(self, name, prob):
        return self.fields[FIELDS_2D[prob.pol].index(name)].reshape(prob.ny, prob.nx)


def run2d(prob, steps=None, state=None, series=False, mutant: int = 0):
    """Runs the 2D oracle on a workloads.Grid2D problem."""
    L = lib(mutant=mutant)
    steps = prob.steps if steps is None else steps
    st = State2D(prob) if state is None else state
    g = OrGrid2D()
    g.nx, g.ny, g.d, g.dt = prob.nx, prob.ny, prob.d, prob.dt
    g.pol = 0 if prob.pol == "tm" else 1
    g.periodic_x = 1 if prob.periodic_x else 0
    g.src_j = prob.src_j
    g.src_tau, g.src_t0, g.src_amp = prob.src_tau, prob.src_t0, prob.src_amp
    g.n_probes, g.n_freq = len(prob.probes), len(prob.freq_hz)
    mat = np.ascontiguousarray(prob.mat, dtype=np.uint8)
    mw = np.ascontiguousarray(prob.mat_wp2, float)
    mn = np.ascontiguousarray(prob.mat_nu, float)
    prof = np.ascontiguousarray(prob.profile, float)
    pr = np.ascontiguousarray(np.asarray(prob.probes, np.int32).ravel() if len(prob.probes) else np.zeros(2, np.int32))
    fr = np.ascontiguousarray(prob.freq_hz, float)
    xr = np.ascontiguousarray(st.X.real.copy())
    xi = np.ascontiguousarray(st.X.imag.copy())
    ser = np.zeros((len(prob.probes), steps)) if series else None
    rc = L.or_run2d(ctypes.byref(g), mat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dp(mw), _dp(mn), len(mw),
                    _dp(prof), pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(fr), st.n, steps,
                    _dp(st.fields), _dp(xr), _dp(xi), _dp(ser) if ser is not None else ctypes.POINTER(ctypes.c_double)())
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    st.X = xr + 1j * xi
    st.n += steps
    return st, ser
