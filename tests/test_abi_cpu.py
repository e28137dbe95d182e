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
    g.bc = {"mur": 0, "cpml": 1, "pml": 2}[slab.bc]
    g.cpml_cells = slab.cpml_cells
    g.cpml_m, g.cpml_sigma_max, g.cpml_kappa_max, g.cpml_alpha_max = rk.CPML_GRADING
    if "grid_prec" in over:
        g.prec = over["grid_prec"]
    if "dt" in over:
        g.dt = over["dt"]
    if "scheme" in over:
        g.scheme = over["scheme"]
    if "bc" in over:
        g.bc = over["bc"]
    opt = None
    if "variant" in over:
        opt = rk.Options()
        L.rketd_default_options(ctypes.byref(opt))
        opt.variant = over["variant"]
    p = rk.Pulse(slab.src_tau, slab.src_t0, slab.src_amp)
    freq = np.ascontiguousarray(slab.freq_hz, float)
    d = rk.Dft(len(slab.probes), len(freq), freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    wp2 = np.ascontiguousarray(slab.wp2, float)
    nu = np.ascontiguousarray(slab.nu, float)
    probes = np.ascontiguousarray(slab.probes, np.int64)
    h = ctypes.c_void_p()
    st = L.rketd_create_1d(slab.nz, ctypes.byref(g), wp2.ctypes.data_as(rk._dp), nu.ctypes.data_as(rk._dp),
                           over.get("src", slab.src_cell), ctypes.byref(p), probes.ctypes.data_as(rk._i64p),
                           ctypes.byref(d), ctypes.byref(opt) if opt is not None else None, None, ctypes.byref(h))
    return st, L.rketd_last_error().decode(), h


def test_courant_above_one_is_rejected():
    s = wl.c1_plain_slab(nz=64, steps=1)
    s.probes = [10, 50]
    st, msg, h = _create(s, dt=1.001 * s.dz * math.sqrt(wl.MU0 * wl.EPS0))
    assert st == 2 and "Courant" in msg and not h.value


@pytest.mark.parametrize("case", ["src0", "src_last", "probe_out", "nu_neg", "wp2_nan", "nz_small", "cpml_thick",
                                  "probe_in_cpml", "bad_prec", "plasma_in_pml", "bad_bc"])
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
    elif case == "plasma_in_pml":
        s.bc, s.cpml_cells = "pml", 5
        s.wp2[3] = 1e20
    elif case == "bad_bc":
        over["bc"] = 3
    st, msg, h = _create(s, **over)
    assert st == 1, (st, msg)
    assert msg and not h.value


@pytest.mark.parametrize("scheme,variant,status", [(3, 0, 1), (-1, 0, 1), (2, 2, 6), (2, 3, 6)])
def test_current_recursion_choices_are_validated_before_any_device_work(scheme, variant, status):
    """An unknown recursion is EINVAL; the Eq. 10 recursion asked of the tiled variant, which does
    not carry E^{n-1}, is EUNSUPPORTED."""
    s = wl.c1_plain_slab(nz=64, steps=1)
    s.src_cell, s.probes = 8, [10, 50]
    st, msg, h = _create(s, scheme=scheme, variant=variant)
    assert st == status, (st, msg)
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


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the ABI structs have the header's sizes and field offsets (gcc)."""
    checks = {"rketd_grid1d": rk.Grid1D, "rketd_grid3d": rk.Grid3D, "rketd_options": rk.Options,
              "rketd_pulse": rk.Pulse, "rketd_dft": rk.Dft}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in checks.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for ln in out:
        if not ln:
            continue
        cname, what, val = ln.split()
        py = checks[cname]
        expect = ctypes.sizeof(py) if what == "size" else getattr(py, what).offset
        assert int(val) == expect, (cname, what)
        seen += 1
    assert seen == sum(len(p._fields_) + 1 for p in checks.values())


def _create3d(prob, **over):
    """Calls rketd_create_3d directly; validation fails before any CUDA call."""
    L = rk.lib()
    g = rk.Grid3D()
    g.nx, g.ny, g.nz, g.prec = prob.nx, prob.ny, prob.nz, over.get("prec", 0)
    g.d, g.dt = prob.d, over.get("dt", prob.dt)
    g.periodic_xy, g.npml = int(prob.periodic_xy), prob.npml
    g.pml_m, g.pml_sigma_max, g.pml_kappa_max, g.pml_alpha_max = rk.CPML_GRADING
    g.tfsf = int(prob.tfsf)
    for q in range(6):
        g.box[q] = prob.box[q]
    g.sheet_k, g.inc_off, g.inc_len, g.inc_src = prob.sheet_k, prob.inc_off, prob.inc_len, prob.inc_src
    mat = np.ascontiguousarray(prob.mat, np.uint8)
    mw = np.ascontiguousarray(over.get("wp2", prob.mat_wp2), float)
    mn = np.ascontiguousarray(prob.mat_nu, float)
    pr = np.ascontiguousarray(np.asarray(prob.probes, np.int32).reshape(-1))
    fr = np.ascontiguousarray(prob.freq_hz, float)
    p = rk.Pulse(prob.src_tau, prob.src_t0, prob.src_amp)
    d = rk.Dft(len(prob.probes), len(fr), fr.ctypes.data_as(rk._dp))
    h = ctypes.c_void_p()
    st = L.rketd_create_3d(ctypes.byref(g), ctypes.c_void_p(mat.ctypes.data), len(mw), mw.ctypes.data_as(rk._dp),
                           mn.ctypes.data_as(rk._dp), ctypes.byref(p), len(prob.probes),
                           ctypes.c_void_p(pr.ctypes.data), ctypes.byref(d), None, ctypes.byref(h))
    return st, L.rketd_last_error().decode(), h


@pytest.mark.parametrize("case", ["courant", "box_in_cpml", "box_empty", "probe_out", "mat0_plasma", "npml_big",
                                  "sheet_in_cpml", "inc_short"])
def test_3d_invalid_inputs_are_rejected_before_any_device_work(case):
    p = wl.sphere_problem(n=32, steps=10, radius=4.0, npml=4, nfreq=4)
    over = {}
    if case == "courant":
        over["dt"] = 1.01 * p.d * math.sqrt(wl.MU0 * wl.EPS0) / math.sqrt(3.0)
    elif case == "box_in_cpml":
        p.box = (3, 20, 8, 20, 8, 20)
    elif case == "box_empty":
        p.box = (10, 10, 8, 20, 8, 20)
    elif case == "probe_out":
        p.probes = [(1, 2, 32)]
    elif case == "mat0_plasma":
        over["wp2"] = np.array([1e20, p.mat_wp2[1]])
    elif case == "npml_big":
        p.npml = 15
    elif case == "sheet_in_cpml":
        p.sheet_k = 2
    elif case == "inc_short":
        p.inc_len = p.nz
    st, msg, h = _create3d(p, **over)
    assert st == (2 if case == "courant" else 1), (st, msg)
    assert msg and not h.value


@pytest.mark.parametrize("case", ["courant", "pol", "src_row", "mat_index", "vacuum0"])
def test_2d_validation_before_any_device_work(case):
    """rketd_create_2d refuses bad input before touching the GPU: runs without one."""
    L = rk.lib()
    nx, ny = 8, 8
    g = rk.Grid2D()
    g.nx, g.ny, g.prec, g.pol, g.d = nx, ny, 0, 0, 1e-4
    g.dt = 0.5 * g.d / wl.C0
    g.periodic_x, g.src_j = 1, 2
    mat = np.zeros(nx * ny, np.uint8)
    wp2 = np.array([0.0, 1e20])
    nu = np.array([0.0, 1e10])
    if case == "courant":
        g.dt = 0.75 * g.d / wl.C0  # above 1/sqrt(2)
    elif case == "pol":
        g.pol = 2
    elif case == "src_row":
        g.src_j = ny - 1
    elif case == "mat_index":
        mat[5] = 2
    elif case == "vacuum0":
        wp2 = np.array([1e20, 1e20])
    prof = np.ones(nx)
    p = rk.Pulse(1e-12, 5e-12, 1.0)
    h = ctypes.c_void_p()
    st = L.rketd_create_2d(ctypes.byref(g), mat.ctypes.data, 2, wp2.ctypes.data_as(rk._dp), nu.ctypes.data_as(rk._dp),
                           prof.ctypes.data_as(rk._dp), ctypes.byref(p), 0, None, None, None, ctypes.byref(h))
    assert st == (2 if case == "courant" else 1), L.rketd_last_error()
    assert not h.value
