"""Pins of the 2D oracle (TMz and TEz, fields uniform along z), CPU only; none uses the oracle to
check itself.

* normal incidence (uniform source profile, periodic x) reduces bit for bit to the 1D oracle along y:
  TMz (Ez, Hx, Jz) = (E, H, J), TEz (Ex, -Hz, Jx) = (E, H, J);
* a single 2D Fourier mode in a uniform medium (vacuum or Drude plasma) keeps its shape and obeys the
  lattice recurrence of Eqs. 11, 12, 14 on rows the Mur ends cannot reach within the run (every x and y
  difference term of both polarisations, to round-off);
* a single transverse mode meeting a plasma layer at oblique incidence (periodic x, Mur y ends) has the
  steady-state R/T of the lattice model (analytic.domain_response_2d_mode: TMz rows q - mu_x; TEz the
  p-polarised rows with Ey half a cell off Ex); the time-domain residual is the finite window's, set
  by a slowly decaying oscillation at the mode's cutoff (measured TEz 1.8e-4, TMz 1.3e-2 at 16000
  steps, for frequencies at least 2.5 times the cutoff);
* planted mistakes in the 2D oracle (a sign, a misplaced material, a shifted difference) fail a pin.
"""
import math

import numpy as np
import pytest

import analytic as an
import oracle
from paper_1709_00821_gb300 import workloads as wl


@pytest.mark.parametrize("pol", ["tm", "te"])
def test_normal_incidence_reduces_bitwise_to_the_1d_oracle(pol):
    p = wl.slab_2d(4, 400, pol, mode=0, steps=1500, d=75e-6)
    st, _ = oracle.run2d(p)
    s1 = wl.Slab1D(p.ny, p.d, p.dt, np.zeros(p.ny), np.zeros(p.ny), p.src_j, p.src_tau, p.src_t0,
                   [p.probes[0][1], p.probes[1][1]], p.freq_hz, "mur", 0, p.steps)
    rows = np.nonzero(p.mat.reshape(p.ny, p.nx)[:, 0])[0]
    s1.wp2[rows] = p.mat_wp2[1]
    s1.nu[rows] = p.mat_nu[1]
    st1, _ = oracle.run1d(s1)
    assert np.abs(st1.J).max() > 0
    E, H, J, sign = ((st.field("Ez", p), st.field("Hx", p), st.field("Jz", p), 1.0) if pol == "tm" else
                     (st.field("Ex", p), st.field("Hz", p), st.field("Jx", p), -1.0))
    for i in range(p.nx):
        assert np.array_equal(E[:, i], st1.E)
        assert np.array_equal(sign * H[:-1, i], st1.H)
        assert np.array_equal(J[:, i], st1.J)
    assert np.array_equal(st.X, st1.X)


def _mode_run(pol, plasma, steps=60, mutant=0):
    """One 2D Fourier mode (kx, ky) = 2 pi (2/16, 3/(ny - 1))-ish on a 16-column periodic grid, uniform
    medium; rows near the middle are out of the Mur ends' reach for `steps` steps."""
    nx, ny = 16, 2 * steps + 12
    wp2, nu = ((2 * math.pi * 30e9) ** 2, 2e10) if plasma else (0.0, 0.0)
    d = 75e-6
    p = wl.Grid2D(nx, ny, d, wl.dt_for_courant(d, 0.5), pol, True, np.full(nx * ny, 1 if plasma else 0, np.uint8),
                  np.array([0.0, wp2]), np.array([0.0, nu]), 1, np.zeros(nx), 1e-12, 5e-12, [], np.array([1e9]),
                  steps, 0.0)
    kx, ky = 2 * math.pi * 2 / nx, 2 * math.pi * 3 / 37
    st = oracle.State2D(p)
    i, j = np.arange(nx)[None, :], np.arange(ny)[:, None]
    F = st.fields.reshape(6, ny, nx)
    if pol == "tm":  # Ez at (i, j)
        F[0] = np.cos(kx * i + ky * j)
        comp = 0
    else:  # Hz at (i + 1/2, j + 1/2)
        F[2] = np.cos(kx * (i + 0.5) + ky * (j + 0.5))
        comp = 2
    mid = slice(ny // 2 - 2, ny // 2 + 3)
    ser = []
    for _ in range(steps):
        ser.append(st.fields.reshape(6, ny, nx)[comp, mid].copy())
        st, _ = oracle.run2d(p, steps=1, state=st, mutant=mutant)
    p1, p2 = an.phi_mp(nu * p.dt)
    a = math.exp(-nu * p.dt)
    w = wp2 * p.dt ** 2
    S = an.courant(d, p.dt)
    A = 2.0 - S * S * (4 * math.sin(kx / 2) ** 2 + 4 * math.sin(ky / 2) ** 2)
    q, pp = w * (p1 - p2), w * p2
    c = np.array([-a - q / 2, 1 + a * A - pp / 2, -(A + a) + q / 2, 1 + pp / 2])  # as for the 3D transverse mode
    ser = np.array(ser)
    res = c[0] * ser[:-3] + c[1] * ser[1:-2] + c[2] * ser[2:-1] + c[3] * ser[3:]
    rec = np.abs(res).max() / (np.abs(ser).max() * np.abs(c).sum())
    pat = ser[0]
    amp = (ser * pat).sum(axis=(1, 2)) / (pat * pat).sum()
    shape = np.abs(ser - amp[:, None, None] * pat).max() / np.abs(ser).max()
    return rec, shape, np.abs(ser).max()


@pytest.mark.parametrize("plasma", [False, True])
@pytest.mark.parametrize("pol", ["tm", "te"])
def test_2d_fourier_mode_obeys_the_lattice_recurrence(pol, plasma):
    rec, shape, peak = _mode_run(pol, plasma)
    assert peak > 0.5
    assert rec <= 1e-14, rec
    assert shape <= 1e-13, shape


def _oblique(pol, steps=16000, mutant=0, nx=64):
    p = wl.slab_2d(nx, 400, pol, mode=1, steps=steps)
    p.src_tau = 5 * p.dt
    p.src_t0 = 5 * p.src_tau
    st, _ = oracle.run2d(p, mutant=mutant)
    sv, _ = oracle.run2d(p.vacuum(), mutant=mutant)
    R, T = oracle.reflection_transmission(st.X, sv.X)
    mu = 4 * math.sin(math.pi / nx) ** 2
    col = p.mat.reshape(p.ny, p.nx)[:, 0]
    rows = [p.probes[0][1], p.probes[1][1]]
    tot = an.domain_response_2d_mode(p.mat_wp2[col], p.mat_nu[col], p.d, p.dt, p.freq_hz, p.src_j, rows, mu, pol)
    inc = an.domain_response_2d_mode(np.zeros(p.ny), np.zeros(p.ny), p.d, p.dt, p.freq_hz, p.src_j, rows, mu, pol)
    Rm, Tm = (tot[:, 0] - inc[:, 0]) / inc[:, 0], tot[:, 1] / inc[:, 1]
    fc = 2 * math.asin(0.5 * math.sin(math.pi / nx)) / (2 * math.pi * p.dt)  # the mode's vacuum cutoff
    band = p.freq_hz >= 2.5 * fc
    return max(np.abs(R - Rm)[band].max(), np.abs(T - Tm)[band].max()), Rm[band], Tm[band]


@pytest.mark.slow
@pytest.mark.parametrize("pol,tol", [("te", 1e-3), ("tm", 3e-2)])
def test_oblique_mode_on_a_plasma_layer_has_the_lattice_response(pol, tol):
    err, Rm, Tm = _oblique(pol)
    assert np.abs(Rm).max() > 0.1 and np.abs(Tm).min() > 0.5  # the layer matters on this band
    assert err <= tol, err


@pytest.mark.parametrize("mutant", [11, 12, 13])
def test_planted_mistakes_in_the_2d_oracle_fail_a_pin(mutant):
    """11: Hy's x term with the wrong sign (TMz); 12: Ey takes the next row's material (TEz);
    13: Hz's x difference at the wrong Ey pair (TEz)."""
    if mutant == 12:
        err, _, _ = _oblique("te", steps=8000, mutant=mutant)
        assert err > 1e-2, err
        return
    pol = "tm" if mutant == 11 else "te"
    rec, shape, _ = _mode_run(pol, True, mutant=mutant)
    assert rec > 1e-10 or shape > 1e-10, (rec, shape)
