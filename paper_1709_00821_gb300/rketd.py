"""Python binding of librketd.so (include/rketd.h): argument marshalling only.

Every numeric step runs in the library's CUDA kernels. The binding loads the
in-tree library and raises if it is missing or if no CUDA device is usable; it
has no fallback path. PyTorch supplies the CUDA stream (and device tensors where
a call takes device pointers).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librketd.so")

RKETD_F32, RKETD_F64 = 0, 1
RKETD_BC_MUR1, RKETD_BC_CPML, RKETD_BC_PML = 0, 1, 2
RKETD_SCHEME_RKETD, RKETD_SCHEME_ETD1, RKETD_SCHEME_ETD2 = 0, 1, 2  # Eq. 11, Eq. 9, Eq. 10
STATUS = {0: "OK", 1: "EINVAL", 2: "ECOURANT", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT", 6: "EUNSUPPORTED",
          7: "ENUMERIC", 8: "EIO"}

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


class RketdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rketd {STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid1D(ctypes.Structure):
    _fields_ = [("dz", ctypes.c_double), ("dt", ctypes.c_double), ("prec", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("cpml_cells", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("cpml_m", ctypes.c_double), ("cpml_sigma_max", ctypes.c_double),
                ("cpml_kappa_max", ctypes.c_double), ("cpml_alpha_max", ctypes.c_double)]


class Pulse(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("t0", ctypes.c_double), ("amp", ctypes.c_double)]


class Dft(ctypes.Structure):
    _fields_ = [("n_probes", ctypes.c_int32), ("n_freq", ctypes.c_int32), ("freq_hz", _dp)]


class Options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("cells_per_lane", ctypes.c_int32), ("tb_steps", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("dft_block", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("fp32_pairs", ctypes.c_int32), ("res_ctas", ctypes.c_int32), ("res_threads", ctypes.c_int32),
                ("res_cells", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class Grid3D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("d", ctypes.c_double), ("dt", ctypes.c_double), ("periodic_xy", ctypes.c_int32),
                ("npml", ctypes.c_int32), ("pml_m", ctypes.c_double), ("pml_sigma_max", ctypes.c_double),
                ("pml_kappa_max", ctypes.c_double), ("pml_alpha_max", ctypes.c_double), ("tfsf", ctypes.c_int32),
                ("box", ctypes.c_int32 * 6), ("sheet_k", ctypes.c_int32), ("inc_off", ctypes.c_int32),
                ("inc_len", ctypes.c_int32), ("inc_src", ctypes.c_int32), ("variant", ctypes.c_int32)]


class Grid2D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("prec", ctypes.c_int32), ("pol", ctypes.c_int32),
                ("d", ctypes.c_double), ("dt", ctypes.c_double), ("periodic_x", ctypes.c_int32),
                ("src_j", ctypes.c_int32)]


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "rketd_default_options": (None, [ctypes.POINTER(Options)]),
    "rketd_create_batch_1d": (ctypes.c_int, [ctypes.c_int32, _i64p, ctypes.POINTER(Grid1D), _dp, _dp, _i64p,
                                             ctypes.POINTER(Pulse), _i64p, ctypes.POINTER(Dft),
                                             ctypes.POINTER(Options), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "rketd_create_1d": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(Grid1D), _dp, _dp, ctypes.c_int64,
                                       ctypes.POINTER(Pulse), _i64p, ctypes.POINTER(Dft), ctypes.POINTER(Options),
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "rketd_set_medium": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "rketd_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "rketd_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_step_index": (ctypes.c_int64, [ctypes.c_void_p]),
    "rketd_get_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _dp, _dp, _dp]),
    "rketd_get_spectra": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "rketd_get_spectra_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rketd_rt": (ctypes.c_int, [_dp, _dp, _dp, _dp, ctypes.c_int32, _dp, _dp, _dp, _dp]),
    "rketd_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "rketd_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "rketd_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rketd_get_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options)]),
    "rketd_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "rketd_check_finite": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int64]),
    "rketd_debug_alloc_count": (ctypes.c_int64, []),
    "rketd_plan_tiles_1d": (ctypes.c_int, [ctypes.c_int32, _i64p, _i64p, ctypes.c_int32, _i64p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i64p, ctypes.c_int64,
                                           _i64p]),
    "rketd_noalloc_tiles_1d": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _i64p, ctypes.c_int64,
                                              _i64p, _i64p]),
    "rketd_kernel_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rketd_get_kernel_timing": (ctypes.c_int, [ctypes.c_void_p, _dp, _i64p, _dp]),
    "rketd_advance_1d_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid1D), ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Pulse),
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "rketd_forward_ckpt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "rketd_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "rketd_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_create_3d": (ctypes.c_int, [ctypes.POINTER(Grid3D), ctypes.c_void_p, ctypes.c_int32, _dp, _dp,
                                       ctypes.POINTER(Pulse), ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Dft),
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "rketd_reset_3d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_step_3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "rketd_get_field_3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _dp]),
    "rketd_get_spectra_3d": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "rketd_kernel_chunk_3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rketd_sync_3d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_launch_count_3d": (ctypes.c_int64, [ctypes.c_void_p]),
    "rketd_set_wait_limit_3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rketd_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rketd_work_3d": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "rketd_check_finite_3d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_destroy_3d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_create_2d": (ctypes.c_int, [ctypes.POINTER(Grid2D), ctypes.c_void_p, ctypes.c_int32, _dp, _dp, _dp,
                                       ctypes.POINTER(Pulse), ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Dft),
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "rketd_reset_2d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_step_2d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "rketd_sync_2d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_get_field_2d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _dp]),
    "rketd_get_spectra_2d": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "rketd_launch_count_2d": (ctypes.c_int64, [ctypes.c_void_p]),
    "rketd_check_finite_2d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_destroy_2d": (ctypes.c_int, [ctypes.c_void_p]),
    "rketd_last_error": (ctypes.c_char_p, []),
    "rketd_version": (ctypes.c_char_p, []),
}


def exported_symbols() -> Sequence[str]:
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """Loads librketd.so (built by __graft_entry__.build()); raises if it is absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(st: int):
    if st != 0:
        raise RketdError(st, lib().rketd_last_error().decode())


def _arr(a, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _default_stream():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the RKETD library runs only on the GPU")
    return torch.cuda.current_stream().cuda_stream


# CPML grading passed to the library: m = 3, sigma_max <= 0 (the library then takes
# 0.8 (m + 1)/(eta0 dz)), kappa_max = 1, alpha_max = 0.05 S/m.
CPML_GRADING = (3.0, 0.0, 1.0, 0.05)


class Context:
    """One rketd_ctx: a batch of 1D slabs advanced together on one CUDA stream."""

    def __init__(self, slabs, prec: str = "f64", options: Optional[dict] = None, stream=None):
        if not isinstance(slabs, (list, tuple)):
            slabs = [slabs]
        L = lib()
        s0 = slabs[0]
        self.slabs = list(slabs)
        self.n_slabs = len(slabs)
        self.n_probes = len(s0.probes)
        self.freq = _arr(s0.freq_hz)
        g = Grid1D()
        g.dz, g.dt = s0.dz, s0.dt
        g.prec = RKETD_F64 if prec == "f64" else RKETD_F32
        g.bc = {"mur": RKETD_BC_MUR1, "cpml": RKETD_BC_CPML, "pml": RKETD_BC_PML}[s0.bc]
        g.cpml_cells = s0.cpml_cells if s0.bc in ("cpml", "pml") else 0
        g.cpml_m, g.cpml_sigma_max, g.cpml_kappa_max, g.cpml_alpha_max = CPML_GRADING
        g.scheme = getattr(s0, "scheme", RKETD_SCHEME_RKETD)
        self.prec = prec
        p = Pulse(s0.src_tau, s0.src_t0, s0.src_amp)
        d = Dft(self.n_probes, len(self.freq), _ptr(self.freq))
        o = Options()
        L.rketd_default_options(ctypes.byref(o))
        for k, v in (options or {}).items():
            setattr(o, k, v)
        nz = _arr([s.nz for s in slabs], np.int64)
        wp2 = _arr(np.concatenate([np.asarray(s.wp2, float) for s in slabs]))
        nu = _arr(np.concatenate([np.asarray(s.nu, float) for s in slabs]))
        src = _arr([s.src_cell for s in slabs], np.int64)
        probes = _arr(np.concatenate([np.asarray(s.probes, np.int64) for s in slabs]) if self.n_probes
                      else np.zeros(1), np.int64)
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _check(L.rketd_create_batch_1d(self.n_slabs, _ptr(nz, _i64p), ctypes.byref(g), _ptr(wp2), _ptr(nu),
                                       _ptr(src, _i64p), ctypes.byref(p), _ptr(probes, _i64p), ctypes.byref(d),
                                       ctypes.byref(o), ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            lib().rketd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def step(self, n: int):
        _check(lib().rketd_step(self.h, int(n)))

    def sync(self):
        _check(lib().rketd_sync(self.h))

    def reset(self):
        _check(lib().rketd_reset(self.h))

    @property
    def step_index(self) -> int:
        return lib().rketd_step_index(self.h)

    def set_medium(self, wp2, nu):
        """Host numpy arrays (copied H2D) or CUDA torch tensors (read on the device), FP64."""
        if hasattr(wp2, "data_ptr"):
            assert wp2.is_cuda and nu.is_cuda and wp2.dtype == nu.dtype
            on_dev = 1
            pw, pn = ctypes.c_void_p(wp2.data_ptr()), ctypes.c_void_p(nu.data_ptr())
        elif isinstance(wp2, int):  # raw device or host pointers
            on_dev = 1
            pw, pn = ctypes.c_void_p(wp2), ctypes.c_void_p(nu)
        else:
            wp2 = _arr(wp2)
            nu = _arr(nu)
            self._keep = (wp2, nu)
            on_dev = 0
            pw, pn = ctypes.c_void_p(wp2.ctypes.data), ctypes.c_void_p(nu.ctypes.data)
        _check(lib().rketd_set_medium(self.h, pw, pn, on_dev))

    def set_medium_host_ptr(self, wp2_ptr: int, nu_ptr: int):
        _check(lib().rketd_set_medium(self.h, ctypes.c_void_p(wp2_ptr), ctypes.c_void_p(nu_ptr), 0))

    def fields(self, slab: int = 0):
        nz = self.slabs[slab].nz
        E, H, J = np.empty(nz), np.empty(nz - 1), np.empty(nz)
        _check(lib().rketd_get_fields(self.h, slab, _ptr(E), _ptr(H), _ptr(J)))
        return E, H, J

    def spectra(self) -> np.ndarray:
        n = self.n_slabs * self.n_probes * len(self.freq)
        re, im = np.empty(n), np.empty(n)
        _check(lib().rketd_get_spectra(self.h, _ptr(re), _ptr(im)))
        return (re + 1j * im).reshape(self.n_slabs, self.n_probes, len(self.freq))

    def spectra_device(self, re_ptr: int, im_ptr: int):
        _check(lib().rketd_get_spectra_device(self.h, ctypes.c_void_p(re_ptr), ctypes.c_void_p(im_ptr)))

    def save(self, path: str):
        _check(lib().rketd_save_state(self.h, path.encode()))

    def load(self, path: str):
        _check(lib().rketd_load_state(self.h, path.encode()))

    def set_wait_limit(self, polls: int):
        """Persistent variant: polls of each neighbour wait (0: every wait gives up; < 0: default)."""
        _check(lib().rketd_set_wait_limit(self.h, int(polls)))

    def autotune(self, passes: int = 8):
        _check(lib().rketd_autotune(self.h, passes))

    def options(self) -> dict:
        o = Options()
        _check(lib().rketd_get_options(self.h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Options._fields_ if k != "reserved"}

    def forward_ckpt(self, nsteps: int, every: int = 512):
        """Reset, run nsteps from rest and keep a state checkpoint every `every` steps."""
        _check(lib().rketd_forward_ckpt(self.h, int(nsteps), int(every)))

    def adjoint(self, gX_re, gX_im, w_lo: int, w_hi: int, grad_wp2, grad_nu):
        """Gradients (into device arrays grad_wp2/grad_nu, FP64, all cells) of a loss whose
        derivatives with respect to the spectra are gX_re/gX_im ([slab, probe, freq], host
        numpy or CUDA tensors)."""
        keep = []

        def ptr(a):
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            arr = _arr(a)
            keep.append(arr)
            return ctypes.c_void_p(arr.ctypes.data)

        _check(lib().rketd_adjoint(self.h, ptr(gX_re), ptr(gX_im), int(w_lo), int(w_hi), ptr(grad_wp2),
                                   ptr(grad_nu)))
        if keep:
            self.sync()

    def kernel_timing(self, enable: bool = True):
        _check(lib().rketd_kernel_timing(self.h, 1 if enable else 0))

    def get_kernel_timing(self):
        """(device ms, launches, cell-updates) of the interior tiled kernel since kernel_timing()."""
        ms, n, cu = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().rketd_get_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(cu)))
        return ms.value, n.value, cu.value

    @property
    def launches(self) -> int:
        return lib().rketd_launch_count(self.h)

    def check_finite(self):
        """Raises RketdError (RKETD_ENUMERIC) if the state or the spectra hold NaN or Inf."""
        _check(lib().rketd_check_finite(self.h))


def rt(tot: np.ndarray, inc: np.ndarray):
    """R, T from [2, n_freq] complex spectra (probe 0 reflection, probe 1 transmission)."""
    n = tot.shape[-1]
    tr, ti = _arr(tot.real), _arr(tot.imag)
    ir, ii = _arr(inc.real), _arr(inc.imag)
    Rr, Ri, Tr, Ti = (np.empty(n) for _ in range(4))
    _check(lib().rketd_rt(_ptr(tr), _ptr(ti), _ptr(ir), _ptr(ii), n, _ptr(Rr), _ptr(Ri), _ptr(Tr), _ptr(Ti)))
    return Rr + 1j * Ri, Tr + 1j * Ti


def advance_1d_noalloc(slab, prec: str, wp2_dev: int, nu_dev: int, n0: int, nsteps: int, E_dev: int, H_dev: int,
                       J_dev: int, stream=None):
    """rketd_advance_1d_noalloc on caller-owned device arrays (raw device pointers, SI units).

    For callers that must not allocate device memory: the library's fixed scratch array
    holds the working state, so nothing is allocated here or in the library call.
    """
    g = Grid1D()
    g.dz, g.dt = slab.dz, slab.dt
    g.prec = RKETD_F64 if prec == "f64" else RKETD_F32
    g.bc = RKETD_BC_MUR1
    g.scheme = getattr(slab, "scheme", RKETD_SCHEME_RKETD)
    p = Pulse(slab.src_tau, slab.src_t0, slab.src_amp)
    st = _default_stream() if stream is None else stream
    _check(lib().rketd_advance_1d_noalloc(ctypes.byref(g), slab.nz, ctypes.c_void_p(wp2_dev), ctypes.c_void_p(nu_dev),
                                          slab.src_cell, ctypes.byref(p), n0, nsteps, ctypes.c_void_p(E_dev),
                                          ctypes.c_void_p(H_dev), ctypes.c_void_p(J_dev), ctypes.c_void_p(st)))


def noalloc_tiles_1d(prec: str, nz: int, src_cell: int):
    """rketd_noalloc_tiles_1d (host only): the no-alloc entry point's tile list as int64 rows (start,
    vlo, vhi, src_local, loaded cells) in launch order, and the tile counts of its three launches."""
    p = RKETD_F64 if prec == "f64" else RKETD_F32
    n = ctypes.c_int64(0)
    counts = np.zeros(3, dtype=np.int64)
    _check(lib().rketd_noalloc_tiles_1d(p, nz, src_cell, None, 0, ctypes.byref(n), _ptr(counts, _i64p)))
    rows = np.zeros((n.value, 5), dtype=np.int64)
    _check(lib().rketd_noalloc_tiles_1d(p, nz, src_cell, _ptr(rows, _i64p), n.value, ctypes.byref(n),
                                        _ptr(counts, _i64p)))
    return rows, counts


FIELDS_3D = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Jx", "Jy", "Jz")


def plan_tiles_1d(nz, src_cell, probe_cell, cpml_cells: int, cells_per_lane: int, tb_steps: int,
                  end_tiles: bool = False) -> np.ndarray:
    """rketd_plan_tiles_1d: the 1D tile plan (host only) as an int64 array of rows (slab, start, vlo,
    vhi, kind, src_local, probe_count, loaded cells), in launch order. probe_cell is [slab][probe]."""
    nz = np.ascontiguousarray(nz, dtype=np.int64)
    src = np.ascontiguousarray(src_cell, dtype=np.int64)
    pc = np.ascontiguousarray(probe_cell, dtype=np.int64).reshape(len(nz), -1)
    n = ctypes.c_int64(0)
    _check(lib().rketd_plan_tiles_1d(len(nz), _ptr(nz, _i64p), _ptr(src, _i64p), pc.shape[1],
                                     _ptr(pc, _i64p) if pc.size else None, cpml_cells, cells_per_lane, tb_steps,
                                     int(end_tiles), None, 0, ctypes.byref(n)))
    rows = np.zeros((n.value, 8), dtype=np.int64)
    _check(lib().rketd_plan_tiles_1d(len(nz), _ptr(nz, _i64p), _ptr(src, _i64p), pc.shape[1],
                                     _ptr(pc, _i64p) if pc.size else None, cpml_cells, cells_per_lane, tb_steps,
                                     int(end_tiles), _ptr(rows, _i64p), n.value, ctypes.byref(n)))
    return rows


class Context3D:
    """One rketd_ctx3d: a 3D Yee RKETD problem (workloads.Grid3D) on one CUDA stream."""

    VARIANTS = {"auto": 0, "plain": 1, "fused": 2, "staged": 3}

    def __init__(self, prob, prec: str = "f32", stream=None, variant: str = "auto", k_chunk: int = 0):
        L = lib()
        self.prob = prob
        g = Grid3D()
        g.nx, g.ny, g.nz = prob.nx, prob.ny, prob.nz
        g.prec = RKETD_F64 if prec == "f64" else RKETD_F32
        g.d, g.dt = prob.d, prob.dt
        g.periodic_xy = 1 if prob.periodic_xy else 0
        g.npml = prob.npml
        g.pml_m, g.pml_sigma_max, g.pml_kappa_max, g.pml_alpha_max = CPML_GRADING
        g.tfsf = 1 if prob.tfsf else 0
        for q in range(6):
            g.box[q] = prob.box[q]
        g.sheet_k = prob.sheet_k
        g.inc_off, g.inc_len, g.inc_src = prob.inc_off, prob.inc_len, prob.inc_src
        g.variant = self.VARIANTS[variant]
        self.prec = prec
        self.n_probes = len(prob.probes)
        self.freq = _arr(prob.freq_hz)
        mat = _arr(prob.mat, np.uint8)
        mw, mn = _arr(prob.mat_wp2), _arr(prob.mat_nu)
        pr = _arr(np.asarray(prob.probes, np.int32).reshape(-1) if self.n_probes else np.zeros(3), np.int32)
        p = Pulse(prob.src_tau, prob.src_t0, prob.src_amp)
        d = Dft(self.n_probes, len(self.freq), _ptr(self.freq))
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _check(L.rketd_create_3d(ctypes.byref(g), ctypes.c_void_p(mat.ctypes.data), len(mw), _ptr(mw), _ptr(mn),
                                 ctypes.byref(p), self.n_probes, ctypes.c_void_p(pr.ctypes.data), ctypes.byref(d),
                                 ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h
        if k_chunk:
            _check(L.rketd_kernel_chunk_3d(self.h, int(k_chunk)))

    def close(self):
        if getattr(self, "h", None):
            lib().rketd_destroy_3d(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int):
        _check(lib().rketd_step_3d(self.h, int(n)))

    def reset(self):
        _check(lib().rketd_reset_3d(self.h))

    def sync(self):
        _check(lib().rketd_sync_3d(self.h))

    def field(self, name: str) -> np.ndarray:
        """One component as a host FP64 SI array [nz, ny, nx]."""
        pb = self.prob
        out = np.empty((pb.nz, pb.ny, pb.nx))
        _check(lib().rketd_get_field_3d(self.h, FIELDS_3D.index(name), _ptr(out)))
        return out

    def spectra(self) -> np.ndarray:
        n = self.n_probes * len(self.freq)
        re, im = np.empty(max(n, 1)), np.empty(max(n, 1))
        _check(lib().rketd_get_spectra_3d(self.h, _ptr(re), _ptr(im)))
        return (re[:n] + 1j * im[:n]).reshape(self.n_probes, len(self.freq))

    @property
    def launches(self) -> int:
        return lib().rketd_launch_count_3d(self.h)

    def check_finite(self):
        """Raises RketdError (RKETD_ENUMERIC) if a field or spectrum holds NaN or Inf."""
        _check(lib().rketd_check_finite_3d(self.h))

    def work(self) -> dict:
        """Tile-planes of each staged work kind (the kinds of the k3_staged kernel's MODE)."""
        v = np.zeros(6, np.int64)
        _check(lib().rketd_work_3d(self.h, v.ctypes.data_as(_i64p)))
        return {name: int(v[k]) for k, name in enumerate(STAGED_KINDS_3D)}

    def set_wait_limit(self, polls: int):
        """Test hook: polls of the staged form's compute-path copy waits (< 0: the default)."""
        _check(lib().rketd_set_wait_limit_3d(self.h, int(polls)))


# work kinds of the 3D staged form, in the order of its kernel's MODE template argument
STAGED_KINDS_3D = ("boundary_xy", "interior_mid", "interior_zc", "boundary_x", "boundary_y", "boundary_faces")

FIELDS_2D = {"tm": ("Ez", "Hx", "Hy", "Jz"), "te": ("Ex", "Ey", "Hz", "Jx", "Jy")}
RKETD_TMZ, RKETD_TEZ = 0, 1


class Context2D:
    """One rketd_ctx2d: a 2D TMz or TEz problem (workloads.Grid2D) on one CUDA stream."""

    def __init__(self, prob, prec: str = "f32", stream=None):
        L = lib()
        self.prob = prob
        g = Grid2D()
        g.nx, g.ny = prob.nx, prob.ny
        g.prec = RKETD_F64 if prec == "f64" else RKETD_F32
        g.pol = RKETD_TMZ if prob.pol == "tm" else RKETD_TEZ
        g.d, g.dt = prob.d, prob.dt
        g.periodic_x = 1 if prob.periodic_x else 0
        g.src_j = prob.src_j
        self.prec = prec
        self.n_probes = len(prob.probes)
        self.freq = _arr(prob.freq_hz)
        mat = _arr(prob.mat, np.uint8)
        mw, mn = _arr(prob.mat_wp2), _arr(prob.mat_nu)
        prof = _arr(prob.profile)
        pr = _arr(np.asarray(prob.probes, np.int32).reshape(-1) if self.n_probes else np.zeros(2), np.int32)
        p = Pulse(prob.src_tau, prob.src_t0, prob.src_amp)
        d = Dft(self.n_probes, len(self.freq), _ptr(self.freq))
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _check(L.rketd_create_2d(ctypes.byref(g), ctypes.c_void_p(mat.ctypes.data), len(mw), _ptr(mw), _ptr(mn),
                                 _ptr(prof), ctypes.byref(p), self.n_probes, ctypes.c_void_p(pr.ctypes.data),
                                 ctypes.byref(d), ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rketd_destroy_2d(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int):
        _check(lib().rketd_step_2d(self.h, int(n)))

    def reset(self):
        _check(lib().rketd_reset_2d(self.h))

    def sync(self):
        _check(lib().rketd_sync_2d(self.h))

    def field(self, name: str) -> np.ndarray:
        """One component as a host FP64 SI array [ny, nx]."""
        out = np.empty((self.prob.ny, self.prob.nx))
        _check(lib().rketd_get_field_2d(self.h, FIELDS_2D[self.prob.pol].index(name), _ptr(out)))
        return out

    def spectra(self) -> np.ndarray:
        n = self.n_probes * len(self.freq)
        re, im = np.empty(max(n, 1)), np.empty(max(n, 1))
        _check(lib().rketd_get_spectra_2d(self.h, _ptr(re), _ptr(im)))
        return (re[:n] + 1j * im[:n]).reshape(self.n_probes, len(self.freq))

    @property
    def launches(self) -> int:
        return lib().rketd_launch_count_2d(self.h)

    def check_finite(self):
        """Raises RketdError (RKETD_ENUMERIC) if a field or spectrum holds NaN or Inf."""
        _check(lib().rketd_check_finite_2d(self.h))


def debug_fail_alloc(after: int):
    """Test hook: the library's device allocation after `after` more successful ones fails as out
    of memory (RKETD_ENOMEM); after < 0 disarms."""
    _check(lib().rketd_debug_fail_alloc(int(after)))


def debug_alloc_count() -> int:
    """Device allocations the library has attempted so far (process-wide)."""
    return lib().rketd_debug_alloc_count()
