"""Parity at the benchmark's full size: the long Epstein slab (2^24 cells, 40000 steps, 512
frequencies, CPML ends), run through the C ABI with the default options that bench.py times.

Nothing reaches further than one cell per step from the source (cell 1032), so after 40000
steps every cell beyond 41034 is still exactly zero, and the cells before it -- probes included
-- are those of the same problem truncated to 41196 cells (its own CPML end beyond the light
cone). The FP64 oracle runs that truncated problem; the GPU runs the full one.
Tolerances: FP64 spectra and fields within 5e-12 of their peak, R/T within 5e-12 of their
peak where the incident spectrum is above 5% of its own peak (measured: 2e-14 .. 4e-13).
FP32: R and T within 1e-4 absolute over that band (measured 7.8e-5 and 4.7e-5; the band edge
divides the FP32 spectra error by 0.05), R within 2e-5 where the incident spectrum is above
half its peak (measured 1.7e-6). Both hold because every carried value is updated by adding
its summed small increment once per step (the folded current of the step kernels); an update
that added da E and dj J to E and J one term at a time lost them below half an ulp and put T
1.7e-4 off on this slab.
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
        # the spectra are within 1e-4 of their peak over the whole band; R and T are held on the
        # 5% band only because they divide that error by the incident spectrum
        assert np.abs(X - tot.X).max() <= 1e-4 * np.abs(tot.X).max()
        assert np.abs(Xv - inc.X).max() <= 1e-4 * np.abs(inc.X).max()
        half = np.abs(inc.X[0]) >= 0.5 * np.abs(inc.X[0]).max()
        errR_half = np.abs(R - Ro)[half].max()
        print(f"FP32: R {errR:.2e}, T {errT:.2e} (absolute, {band.sum()} of {band.size} frequencies); "
              f"R {errR_half:.2e} where the source is above half its peak")
        assert errR_half <= 2e-5
        assert errR <= 1e-4 and errT <= 1e-4


def _c4_loss(X, Xi, tgt):
    """Loss sum_f (|R(f)| - |R_t(f)|)^2 with R = (X - X_inc)/X_inc at the reflection probe, and its
    derivatives with respect to Re X and Im X."""
    d = X - Xi
    absr = np.abs(d) / np.abs(Xi)
    loss = float(np.sum((absr - tgt) ** 2))
    coef = 2 * (absr - tgt) / (np.abs(Xi) * np.abs(d))
    return loss, coef * d.real, coef * d.imag


def test_full_size_adjoint_gradient_matches_central_differences():
    """Adjoint workload at full size (65536-cell lines, 30000 steps, checkpoint every 512, window
    [2048, 6144), 256 frequencies, two profiles batched). The oracle's adjoint keeps the whole
    field history, which this size does not allow, so the FP64 gradient is checked by the
    property that holds at any size: its directional derivative equals the central difference of
    the loss along a smooth random direction (FP64 forward runs). The FP32 gradient of the
    benchmark's precision is then checked against it, 1e-3 relative in norm."""
    import os

    import torch

    tgt = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "c4_target.txt"))[:, 1]
    profs = [wl.c4_profile(i) for i in range(2)]
    steps, every, (lo, hi) = profs[0].steps, 512, (2048, 6144)
    with rk.Context(profs[0].vacuum(), "f64") as cv:
        cv.step(steps)
        Xi = cv.spectra()[0, 0]
    n = sum(p.nz for p in profs)

    def loss_of(ps, prec):
        with rk.Context(ps, prec) as c:
            c.step(steps)
            X = c.spectra()[:, 0]
        return sum(_c4_loss(X[s], Xi, tgt)[0] for s in range(len(ps)))

    def grad(prec):
        with rk.Context(profs, prec) as c:
            c.forward_ckpt(steps, every)
            X = c.spectra()[:, 0]
            gX = np.zeros((len(profs), 1, X.shape[1]), complex)
            for s in range(len(profs)):
                _, gr, gi = _c4_loss(X[s], Xi, tgt)
                gX[s, 0] = gr + 1j * gi
            gw = torch.empty(n, dtype=torch.float64, device="cuda")
            gn = torch.empty(n, dtype=torch.float64, device="cuda")
            c.adjoint(np.ascontiguousarray(gX.real), np.ascontiguousarray(gX.imag), lo, hi, gw, gn)
            c.sync()
            return gw.cpu().numpy(), gn.cpu().numpy()

    gw64, gn64 = grad("f64")
    # smooth random direction inside the window, relative to each profile's own values
    u = (np.arange(hi - lo) + 0.5) / (hi - lo)
    r1 = wl.uniform01(0x5EED01, 8) - 0.5
    r2 = wl.uniform01(0x5EED02, 8) - 0.5
    shape1 = sum(r1[m] * np.sin((m + 1) * np.pi * u) for m in range(8))
    shape2 = sum(r2[m] * np.sin((m + 1) * np.pi * u) for m in range(8))
    h = 1e-5
    vw = np.zeros(n)
    vn = np.zeros(n)
    for s, p in enumerate(profs):
        off = s * p.nz
        vw[off + lo:off + hi] = p.wp2[lo:hi] * shape1
        vn[off + lo:off + hi] = p.nu[lo:hi] * shape2
    directional = float(np.dot(gw64, vw) + np.dot(gn64, vn))

    def moved(sign):
        out = []
        for s, p in enumerate(profs):
            q = wl.Slab1D(p.nz, p.dz, p.dt, p.wp2 + sign * h * vw[s * p.nz:(s + 1) * p.nz],
                          p.nu + sign * h * vn[s * p.nz:(s + 1) * p.nz], p.src_cell, p.src_tau, p.src_t0,
                          list(p.probes), p.freq_hz, p.bc, p.cpml_cells, p.steps, p.src_amp)
            out.append(q)
        return out

    fd = (loss_of(moved(+1), "f64") - loss_of(moved(-1), "f64")) / (2 * h)
    rel = abs(fd - directional) / abs(directional)
    print(f"FP64 adjoint: directional derivative {directional:.9e}, central difference {fd:.9e}, rel {rel:.2e}")
    assert rel <= 1e-6
    gw32, gn32 = grad("f32")
    win = np.zeros(n, bool)
    for s, p in enumerate(profs):
        win[s * p.nz + lo:s * p.nz + hi] = True
    e_w = np.linalg.norm(gw32[win] - gw64[win]) / np.linalg.norm(gw64[win])
    e_n = np.linalg.norm(gn32[win] - gn64[win]) / np.linalg.norm(gn64[win])
    print(f"FP32 adjoint vs FP64: wp2 {e_w:.2e}, nu {e_n:.2e} (relative, norm over the window)")
    assert e_w <= 1e-3 and e_n <= 1e-3
    assert not np.any(gw32[~win]) and not np.any(gn32[~win])
