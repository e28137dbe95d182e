"""C-ABI checks that need no GPU: exports, header coverage, host-side validation."""
import ctypes
import math
import re
import subprocess

import numpy as np
import pytest

from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

HEADER = rk.HERE + "/../include/rketd.h"


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(rketd_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_entry_point():
    L = rk.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", rk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rketd_\w+)", out))
    assert set(names) <= exported
    assert set(rk.exported_symbols()) <= set(names)


def _create(slab, prec="f64", **over):
    """Calls rketd_create_1d directly with stream 0; validation fails before any CUDA call."""
    L = rk.lib()
    g = rk.Grid1D()
    g.dz, g.dt = slab.dz, slab.dt
    g.prec = 1 if prec == "f64" else 0
    g.bc = 1 if slab.bc == "cpml" else 0
    g.cpml_cells = slab.cpml_cells
    g.cpml_m, g.cpml_sigma_max, g.cpml_kappa_max, g.cpml_alpha_max = rk.cpml_params(slab.dz)
    if "grid_prec" in over:
        g.prec = over["grid_prec"]
    if "dt" in over:
        g.dt = over["dt"]
    p = rk.Pulse(slab.src_tau, slab.src_t0, slab.src_amp)
    freq = np.ascontiguousarray(slab.freq_hz, float)
    d = rk.Dft(len(slab.probes), len(freq), freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    wp2 = np.ascontiguousarray(slab.wp2, float)
    nu = np.ascontiguousarray(slab.nu, float)
    probes = np.ascontiguousarray(slab.probes, np.int64)
    h = ctypes.c_void_p()
    st = L.rketd_create_1d(slab.nz, ctypes.byref(g), wp2.ctypes.data_as(rk._dp), nu.ctypes.data_as(rk._dp),
                           over.get("src", slab.src_cell), ctypes.byref(p), probes.ctypes.data_as(rk._i64p),
                           ctypes.byref(d), None, None, ctypes.byref(h))
    return st, L.rketd_last_error().decode(), h


def test_courant_above_one_is_rejected():
    s = wl.c1_plain_slab(nz=64, steps=1)
    s.probes = [10, 50]
    st, msg, h = _create(s, dt=1.001 * s.dz * math.sqrt(wl.MU0 * wl.EPS0))
    assert st == 2 and "Courant" in msg and not h.value


@pytest.mark.parametrize("case", ["src0", "src_last", "probe_out", "nu_neg", "wp2_nan", "nz_small", "cpml_thick",
                                  "probe_in_cpml", "bad_prec"])
def test_invalid_inputs_are_rejected_before_any_device_work(case):
    s = wl.c1_plain_slab(nz=64, steps=1)
    s.src_cell, s.probes = 8, [10, 50]
    over = {}
    if case == "src0":
        over["src"] = 0
    elif case == "src_last":
        over["src"] = 63
    elif case == "probe_out":
        s.probes = [10, 64]
    elif case == "nu_neg":
        s.nu[5] = -1.0
    elif case == "wp2_nan":
        s.wp2[5] = np.nan
    elif case == "nz_small":
        s = wl.c1_plain_slab(nz=7, steps=1)
        s.src_cell, s.probes = 2, [1, 5]
    elif case == "cpml_thick":
        s.bc, s.cpml_cells = "cpml", 31
    elif case == "probe_in_cpml":
        s.bc, s.cpml_cells = "cpml", 12
        s.probes = [5, 40]
    elif case == "bad_prec":
        over["grid_prec"] = 7
    st, msg, h = _create(s, **over)
    assert st == 1, (st, msg)
    assert msg and not h.value


def test_rt_helper_divides_spectra():
    rng = np.random.default_rng(0)
    tot = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    inc = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    R, T = rk.rt(tot, inc)
    assert np.allclose(R, (tot[0] - inc[0]) / inc[0], rtol=1e-15, atol=0)
    assert np.allclose(T, tot[1] / inc[1], rtol=1e-15, atol=0)


def test_rt_helper_reports_zero_incident_spectrum():
    tot = np.ones((2, 3), complex)
    inc = np.ones((2, 3), complex)
    inc[0, 1] = 0
    with pytest.raises(rk.RketdError) as ei:
        rk.rt(tot, inc)
    assert ei.value.status == 7
