"""Pins of the oracle's other two current recursions (CPU only): the first-order ETD of Eq. 9 and
Eq. 10 read literally (F extrapolated from F_{n-1} and F_n over the step, an explicit second-order
ETD), beside the RKETD recursion of Eq. 11 that the rest of the library implements.

* each scheme's running-DFT R/T converge to the steady-state response of its own lattice
  (analytic.domain_rt with that scheme's discrete permittivity), which differs between schemes by
  far more than the convergence residual, so the pin tells the schemes apart;
* one step from a random state satisfies Eq. 9 or Eq. 10 and Eq. 12 in 40-digit arithmetic;
* with wp = 0 every scheme is the textbook Yee loop bit for bit; a resumed run is bitwise equal;
* a planted sign mistake in Eq. 10 fails the lattice pin;
* the accuracy order: on the lattice, the slab's |R| and |T| approach the continuous (Airy) slab
  as the grid is refined at fixed Courant number with error ratios 4 (Eq. 11 and Eq. 10, second
  order) and 2 (Eq. 9, first order) per halving.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import analytic as an
import oracle
from paper_1709_00821_gb300 import workloads as wl

SCHEMES = {1: "Eq. 9", 2: "Eq. 10"}


def _slab(scheme, **kw):
    s = wl.c1_plain_slab(**kw)
    s.scheme = scheme
    return s


def _rt(slab, **kw):
    st, _ = oracle.run1d(slab, **kw)
    sv, _ = oracle.run1d(slab.vacuum(), **kw)
    return oracle.reflection_transmission(st.X, sv.X)


@pytest.fixture(scope="module")
def lattice():
    return {k: an.domain_rt(_slab(k)) for k in (0, 1, 2)}


@pytest.mark.parametrize("scheme", [1, 2])
def test_each_scheme_converges_to_its_own_finite_lattice_response(scheme, lattice):
    Rd, Td = lattice[scheme]
    R8, T8 = _rt(_slab(scheme, steps=8000))
    R16, T16 = _rt(_slab(scheme, steps=16000))
    e8 = max(np.abs(R8 - Rd).max(), np.abs(T8 - Td).max())
    e16 = max(np.abs(R16 - Rd).max(), np.abs(T16 - Td).max())
    assert e16 < 1e-4 and e16 < e8 / 50, (e8, e16)
    hi = slice(70, None)  # >= 35.5 GHz
    assert max(np.abs(R16 - Rd)[hi].max(), np.abs(T16 - Td)[hi].max()) < 1e-7
    # the schemes' lattices differ by far more than the residual (measured 4e-2 for Eq. 9, 2.4e-3 for Eq. 10)
    R0, T0 = lattice[0]
    assert max(np.abs(Rd - R0).max(), np.abs(Td - T0).max()) > 1e-3


@pytest.mark.parametrize("scheme", [1, 2])
def test_single_step_satisfies_the_current_recursion_and_eq_12(scheme):
    nz = 48
    s = _slab(scheme, nz=nz, steps=1)
    s.src_amp = 0.0
    u = wl.uniform01(21, 4 * nz)
    s.wp2 = (2 * math.pi * 60e9 * u[:nz]) ** 2
    s.nu = 1e11 * u[nz:2 * nz]
    st0 = oracle.State1D(s)
    g = wl.normal(22, 4 * nz)
    jscale = an.EPS0 / s.dt
    st0.E[:] = g[:nz]
    st0.H[:] = g[nz:2 * nz - 1] / math.sqrt(an.MU0 / an.EPS0)
    st0.J[:] = g[2 * nz:3 * nz] * jscale
    st0.Eprev[:] = g[3 * nz:]
    st0.n = 41
    st1, _ = oracle.run1d(s, state=st0.copy())
    mp.mp.dps = 40
    M = lambda x: mp.mpf(float(x))
    dt, dz = M(s.dt), M(s.dz)
    eps0 = M(an.EPS0)
    worst = {"J": 0.0, "12": 0.0}
    for k in range(1, nz - 1):
        nu = M(s.nu[k])
        x = nu * dt
        a = mp.exp(-x)
        F = lambda e: eps0 * M(s.wp2[k]) * M(e)
        rhs = a * M(st0.J[k]) + (1 - a) / nu * F(st0.E[k])  # Eq. 9
        terms = [abs(a * M(st0.J[k])), abs((1 - a) / nu * F(st0.E[k]))]
        if scheme == 2:  # Eq. 10: + (e^{-nu dt} - 1 + nu dt)/(nu^2 dt) (F_n - F_{n-1})
            extra = (a - 1 + x) / (nu ** 2 * dt) * (F(st0.E[k]) - F(st0.Eprev[k]))
            rhs += extra
            terms.append(abs(extra))
        worst["J"] = max(worst["J"], float(abs(M(st1.J[k]) - rhs) / max(terms + [abs(rhs)])))
        curl = dt / (eps0 * dz) * (M(st1.H[k]) - M(st1.H[k - 1]))
        rhs = M(st0.E[k]) - curl - dt / (2 * eps0) * (M(st1.J[k]) + M(st0.J[k]))
        sc = max(abs(M(st0.E[k])), abs(curl), abs(rhs))
        worst["12"] = max(worst["12"], float(abs(M(st1.E[k]) - rhs) / sc))
    assert worst["J"] < 1e-14 and worst["12"] < 1e-14, worst
    if scheme == 2:  # the carried E^{n-1} is now E^n
        assert np.array_equal(st1.Eprev[1:-1], st0.E[1:-1])


@pytest.mark.parametrize("scheme", [1, 2])
def test_zero_plasma_frequency_is_bitwise_plain_yee_and_resume_is_bitwise(scheme):
    s = _slab(scheme, nz=600, steps=900).vacuum()
    s.src_cell, s.probes = 200, [100, 500]
    st, ser = oracle.run1d(s, series=True)
    src = lambda t: s.src_amp * ((t - s.src_t0) / s.src_tau) * math.exp(-0.5 * ((t - s.src_t0) / s.src_tau) ** 2)
    E, H, ser_y = an.plain_yee_vacuum(s.nz, s.dz, s.dt, s.steps, s.src_cell, src, s.probes)
    assert np.array_equal(st.E, E) and np.array_equal(st.H, H) and np.array_equal(ser, ser_y)
    p = _slab(scheme, steps=700)
    a, _ = oracle.run1d(p)
    b, _ = oracle.run1d(p, steps=300)
    b, _ = oracle.run1d(p, steps=400, state=b)
    for f in ("E", "H", "J", "Eprev", "X"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_planted_sign_mistake_in_eq_10_fails_the_lattice_pin(lattice):
    Rd, Td = lattice[2]
    R, T = _rt(_slab(2, steps=16000), mutant=9)
    hi = slice(70, None)
    assert max(np.abs(R - Rd)[hi].max(), np.abs(T - Td)[hi].max()) > 1e-5


def test_accuracy_order_of_the_three_recursions_on_the_lattice():
    """|R| and |T| of the paper's 9 mm slab (wp = 2 pi 28.7 GHz, nu = 2e10) on the infinite lattice
    against the continuous slab at 5..60 GHz, grid refined 150 -> 9.4 um at Courant 0.5. The lattice
    permittivity of each scheme is the one the previous tests pin the oracle to. Measured ratios:
    4.00-4.02 (Eq. 11), 2.01-2.05 (Eq. 9), 4.01-4.05 (Eq. 10)."""
    freqs = np.array([5e9, 10e9, 20e9, 30e9, 40e9, 60e9])
    wp2, nu, d = (2 * math.pi * 28.7e9) ** 2, 2e10, 9e-3
    Rf, Tf = an.fresnel_slab(freqs, wp2, nu, d)
    errs = {}
    for scheme in (0, 1, 2):
        e = []
        for dz in (150e-6, 75e-6, 37.5e-6, 18.75e-6, 9.375e-6):
            n = int(round(d / dz))
            nz = n + 40
            w = np.zeros(nz)
            v = np.zeros(nz)
            w[20:20 + n] = wp2
            v[20:20 + n] = nu
            R, T = an.slab_rt_lattice(w, v, dz, wl.dt_for_courant(dz, 0.5), freqs, 10, nz - 10, scheme)
            e.append(max(np.abs(np.abs(R) - Rf).max(), np.abs(np.abs(T) - Tf).max()))
        errs[scheme] = np.array(e)
    for scheme, (lo, hi) in ((0, (3.8, 4.2)), (1, (1.9, 2.1)), (2, (3.8, 4.2))):
        r = errs[scheme][:-1] / errs[scheme][1:]
        assert np.all((r > lo) & (r < hi)), (scheme, r)
    # at every resolution the first-order scheme is the least accurate
    assert np.all(errs[1] > 10 * errs[0]) and np.all(errs[1] > 10 * errs[2])
