"""Parity at the benchmark's full size: the long Epstein slab (2^24 cells, 40000 steps, 512
frequencies, CPML ends), run through the C ABI with the default options that bench.py times.

Nothing reaches further than one cell per step from the source (cell 1032), so after 40000
steps every cell beyond 41034 is still exactly zero, and the cells before it -- probes included
-- are those of the same problem truncated to 41196 cells (its own CPML end beyond the light
cone). The FP64 oracle runs that truncated problem; the GPU runs the full one.
Tolerances: FP64 spectra and fields within 5e-12 of their peak, R/T within 5e-12 of their
peak where the incident spectrum is above 5% of its own peak (measured: 5e-14 .. 4e-13).
FP32: R within 1e-4 absolute where the incident spectrum is above half its peak (measured
4.3e-5); over the 5% band R and T within 2.5e-4 (measured 1.6e-4 and 1.7e-4). The 1e-4 bar
for FP32 R/T holds on the 8000-step slab of Sec. IV.B; on this 40000-step slab the
transmission probe sits 12 mm inside the plasma and the rounding of the FP32 fields alone
(every other step in FP64 or compensated) puts the FP32 spectra 1.5e-4 from the FP64 oracle
there, so T misses it by 1.7x.
"""
import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _truncated(s, n):
    t = wl.Slab1D(n, s.dz, s.dt, s.wp2[:n].copy(), s.nu[:n].copy(), s.src_cell, s.src_tau, s.src_t0,
                  list(s.probes), s.freq_hz, s.bc, s.cpml_cells, s.steps, s.src_amp)
    return t


@pytest.fixture(scope="module")
def c2():
    s = wl.c2_epstein()
    reach = s.src_cell + s.steps + 2
    t = _truncated(s, reach + 2 * s.cpml_cells + 100)
    tot, _ = oracle.run1d(t, omp=True)
    inc, _ = oracle.run1d(t.vacuum(), omp=True)
    return s, reach, tot, inc


def _gpu(s, prec):
    with rk.Context(s, prec) as ctx:
        ctx.step(s.steps)
        X = ctx.spectra()[0]
        E, H, J = ctx.fields(0)
    return X, E, H, J


def _band(inc):
    mag = np.abs(inc.X[0])
    return mag >= 0.05 * mag.max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_epstein_slab_matches_the_oracle_inside_the_light_cone(c2, prec):
    s, reach, tot, inc = c2
    X, E, H, J = _gpu(s, prec)
    Xv, Ev, _, _ = _gpu(s.vacuum(), prec)
    # beyond the light cone nothing has moved, bit for bit
    assert not np.any(E[reach:]) and not np.any(H[reach:]) and not np.any(J[reach:])
    assert not np.any(Ev[reach:])
    n = tot.E.size
    R, T = rk.rt(X, Xv)
    Ro, To = oracle.reflection_transmission(tot.X, inc.X)
    band = _band(inc)
    errR = np.abs(R - Ro)[band].max()
    errT = np.abs(T - To)[band].max()
    if prec == "f64":
        eX = np.abs(X - tot.X).max() / np.abs(tot.X).max()
        eE = np.abs(E[:n] - tot.E).max() / np.abs(tot.E).max()
        print(f"FP64: spectra {eX:.2e}, fields {eE:.2e}, R {errR / np.abs(Ro).max():.2e}, "
              f"T {errT / np.abs(To).max():.2e}")
        assert eX <= 5e-12 and eE <= 5e-12
        assert errR <= 5e-12 * np.abs(Ro).max() and errT <= 5e-12 * np.abs(To).max()
    else:
        half = np.abs(inc.X[0]) >= 0.5 * np.abs(inc.X[0]).max()
        errR_half = np.abs(R - Ro)[half].max()
        print(f"FP32: R {errR:.2e}, T {errT:.2e} (absolute, {band.sum()} of {band.size} frequencies); "
              f"R {errR_half:.2e} where the source is above half its peak")
        assert errR_half <= 1e-4
        assert errR <= 2.5e-4 and errT <= 2.5e-4
