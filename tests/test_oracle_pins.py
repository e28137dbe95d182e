"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the property it checks; together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them (the planted-mistake test shows it for four such
mistakes).
"""
import math

import mpmath as mp
import numpy as np
import pytest

import analytic as an
import oracle
from paper_1709_00821_gb300 import workloads as wl


def _rt(slab, **kw):
    st, _ = oracle.run1d(slab, **kw)
    sv, _ = oracle.run1d(slab.vacuum(), **kw)
    return oracle.reflection_transmission(st.X, sv.X)


@pytest.fixture(scope="module")
def c1_exact():
    return an.domain_rt(wl.c1_plain_slab())


@pytest.fixture(scope="module")
def c1_16k():
    return _rt(wl.c1_plain_slab(steps=16000))


def test_phi_series_and_expm1_branches_match_40_digit_values():
    """phi1, phi2 (the Eq. 7 -> Eq. 11 integrals) against mpmath, both sides of the series switch."""
    xs = [0.0, 1e-12, 1.7e-6, 8.3e-5, 2.5e-3, 1.25e-2, 0.1, 0.5, 0.9999999, 1.0, 1.0000001, 3.0, 30.0]
    for x in xs:
        p1, p2 = an.phi_mp(x)
        assert abs(oracle.phi1(x) - p1) <= 5e-16 * abs(p1), x
        assert abs(oracle.phi2(x) - p2) <= 5e-16 * abs(p2), x


def test_rt_converges_to_exact_finite_lattice_response(c1_exact, c1_16k):
    """P1: the running-DFT R/T converge to the lattice's own steady-state response (Mur ends included)."""
    Rd, Td = c1_exact
    R8, T8 = _rt(wl.c1_plain_slab(steps=8000))
    R16, T16 = c1_16k
    e8 = max(np.abs(R8 - Rd).max(), np.abs(T8 - Td).max())
    e16 = max(np.abs(R16 - Rd).max(), np.abs(T16 - Td).max())
    assert e8 < 5e-3
    assert e16 < 1e-4
    assert e16 < e8 / 50  # the residual is window truncation: it shrinks with the window
    hi = slice(70, None)  # >= 35.5 GHz, where the fields have decayed by 16000 steps
    assert np.abs(R16 - Rd)[hi].max() < 1e-7
    assert np.abs(T16 - Td)[hi].max() < 1e-7


def test_rt_near_infinite_lattice_transfer_matrix(c1_16k):
    """P1 (slab alone): transfer recursion on the infinite lattice; differs only by the Mur ends."""
    s = wl.c1_plain_slab()
    Rl, Tl = an.slab_rt_lattice(s.wp2, s.nu, s.dz, s.dt, s.freq_hz, 300, 1700)
    R16, T16 = c1_16k
    assert np.abs(R16 - Rl).max() < 3e-3
    assert np.abs(T16 - Tl).max() < 3e-3


def test_rt_magnitudes_match_continuous_fresnel_slab():
    """P2: |R|, |T| within 1e-2 of the Airy slab with eps_r = 1 - wp^2/(w(w - j nu)), 0.5-100 GHz."""
    s = wl.c1_plain_slab()
    R, T = _rt(s)
    Rf, Tf = an.fresnel_slab(s.freq_hz, s.wp2[850], s.nu[850], 120 * s.dz)
    assert np.abs(np.abs(R) - Rf).max() <= 1e-2
    assert np.abs(np.abs(T) - Tf).max() <= 1e-2


def test_zero_plasma_frequency_is_bitwise_plain_yee():
    """P3: with wp = 0 the scheme is the plain Yee leapfrog, bit for bit, whatever nu is."""
    s = wl.c1_plain_slab(nz=600, steps=900)
    s.src_cell, s.probes = 100, [200, 400]
    s.wp2[:] = 0.0
    s.nu[:] = wl.uniform01(7, s.nz) * 1e11
    st, ser = oracle.run1d(s, series=True)
    E, H, ser_y = an.plain_yee_vacuum(s.nz, s.dz, s.dt, s.steps, s.src_cell,
                                      lambda t: s.src_amp * ((t - s.src_t0) / s.src_tau)
                                      * math.exp(-0.5 * ((t - s.src_t0) / s.src_tau) ** 2), s.probes)
    assert np.array_equal(st.E, E)
    assert np.array_equal(st.H, H)
    assert np.array_equal(ser, ser_y)
    assert not np.any(st.J)
    sv, _ = oracle.run1d(s.vacuum())
    assert np.array_equal(st.X, sv.X)  # total == incident spectra: R = 0 and T = 1 exactly


def test_lossless_plasma_conserves_energy_and_lossy_plasma_does_not_gain():
    """P4: nu = 0 gives |R|^2 + |T|^2 = 1 (up to Mur and window); nu > 0 gives <= 1 at every f."""
    s0 = wl.c1_plain_slab(steps=16000, nu=0.0)
    R, T = _rt(s0)
    bal = np.abs(R) ** 2 + np.abs(T) ** 2
    assert np.abs(bal - 1).max() < 1e-3
    Rl, Tl = an.slab_rt_lattice(s0.wp2, s0.nu, s0.dz, s0.dt, s0.freq_hz, 300, 1700)
    assert np.abs(np.abs(Rl) ** 2 + np.abs(Tl) ** 2 - 1).max() < 1e-11  # lossless lattice, exact
    R1, T1 = _rt(wl.c1_plain_slab(steps=16000))
    assert np.all(np.abs(R1) ** 2 + np.abs(T1) ** 2 <= 1 + 1e-4)


def test_magic_time_step_translates_one_cell_per_step_and_mur_absorbs():
    """P5: at S = 1 vacuum pulses move exactly one cell per step and first-order Mur is exact.

    Initial state: a right-going pulse f1 and a left-going pulse f2 (normalised H~ = eta0 H),
    E_k = f1(k) + f2(k), H~_{k+1/2} = f1(k+1) - f2(k), so that E^n_k = f1(k-n) + f2(k+n).
    """
    dz = 75e-6
    dt = dz * math.sqrt(an.MU0 * an.EPS0)
    nz = 400
    s = wl.c1_plain_slab(nz=nz, steps=700)
    s.dt = dt
    s.src_amp = 0.0
    s.wp2[:] = 0.0
    s.nu[:] = 0.0
    s.src_cell, s.probes = 50, [200, 300]
    f1 = lambda x: np.exp(-((x - 120.0) / 9.0) ** 2)
    f2 = lambda x: -0.5 * np.exp(-((x - 260.0) / 6.0) ** 2)
    k = np.arange(nz, dtype=float)
    st0 = oracle.State1D(s)
    st0.E[:] = f1(k) + f2(k)
    st0.H[:] = (f1(k[:-1] + 1) - f2(k[:-1])) / math.sqrt(an.MU0 / an.EPS0)
    st, ser = oracle.run1d(s, state=st0, series=True)
    n = np.arange(1, s.steps + 1)
    for p, cell in enumerate(s.probes):
        assert np.abs(ser[p] - (f1(cell - n) + f2(cell + n))).max() <= 1e-12
    assert np.abs(st.E).max() <= 1e-12  # both pulses left through the Mur ends


def test_courant_above_one_diverges_below_one_stays_bounded():
    """P5: S = 1.01 amplifies round-off exponentially; S = 0.99 stays bounded."""
    out = {}
    for S in (0.99, 1.01):
        s = wl.c1_plain_slab(nz=400, steps=600)
        s.dt = S * s.dz * math.sqrt(an.MU0 * an.EPS0)
        s.src_tau = 15 * s.dt
        s.src_t0 = 5 * s.src_tau
        s.wp2[:] = 0.0
        s.src_cell, s.probes = 50, [200, 300]
        with np.errstate(all="ignore"):
            st, _ = oracle.run1d(s)
        m = np.nanmax(np.abs(st.E)) if np.all(np.isfinite(st.E)) else np.inf
        out[S] = m
    assert out[0.99] < 2.0
    assert out[1.01] > 1e6


def test_single_step_satisfies_eqs_11_12_14():
    """P6: one oracle step from a random state satisfies Eqs. 14, 12 and 11 to rounding."""
    nz = 48
    s = wl.c1_plain_slab(nz=nz, steps=1)
    s.src_amp = 0.0
    u = wl.uniform01(11, 4 * nz)
    s.wp2 = (2 * math.pi * 60e9 * u[:nz]) ** 2
    s.nu = 1e11 * u[nz:2 * nz]
    st0 = oracle.State1D(s)
    g = wl.normal(12, 3 * nz)
    jscale = an.EPS0 / s.dt
    st0.E[:] = g[:nz]
    st0.H[:] = g[nz:2 * nz - 1] / math.sqrt(an.MU0 / an.EPS0)
    st0.J[:] = g[2 * nz:] * jscale
    st0.n = 37
    st1, _ = oracle.run1d(s, state=st0.copy())
    mp.mp.dps = 40
    M = lambda x: mp.mpf(float(x))
    dt, dz = M(s.dt), M(s.dz)
    eps0, mu0 = M(an.EPS0), M(an.MU0)
    worst = {"14": 0.0, "12": 0.0, "11": 0.0}
    for k in range(nz - 1):
        rhs = M(st0.H[k]) - dt / (mu0 * dz) * (M(st0.E[k + 1]) - M(st0.E[k]))
        sc = max(abs(M(st0.H[k])), abs(rhs))
        worst["14"] = max(worst["14"], float(abs(M(st1.H[k]) - rhs) / sc))
    for k in range(1, nz - 1):
        rhs = (M(st0.E[k]) - dt / (eps0 * dz) * (M(st1.H[k]) - M(st1.H[k - 1]))
               - dt / (2 * eps0) * (M(st1.J[k]) + M(st0.J[k])))
        sc = max(abs(M(st0.E[k])), abs(dt / (eps0 * dz) * (M(st1.H[k]) - M(st1.H[k - 1]))), abs(rhs))
        worst["12"] = max(worst["12"], float(abs(M(st1.E[k]) - rhs) / sc))
        x = M(s.nu[k]) * dt
        a = mp.exp(-x)
        wp2 = M(s.wp2[k])
        b1 = eps0 * wp2 * (1 - a) / M(s.nu[k])
        b2 = eps0 * wp2 * (a - 1 + x) / (M(s.nu[k]) ** 2 * dt)
        rhs = a * M(st0.J[k]) + b1 * M(st0.E[k]) + b2 * (M(st1.E[k]) - M(st0.E[k]))
        sc = max(abs(a * M(st0.J[k])), abs(b1 * M(st0.E[k])), abs(rhs))
        worst["11"] = max(worst["11"], float(abs(M(st1.J[k]) - rhs) / sc))
    assert worst["14"] < 1e-15 and worst["12"] < 1e-14 and worst["11"] < 1e-14, worst


def test_cpml_reflection_below_1e4_of_incident_peak():
    """P7: a 32-cell CPML (m = 3, sigma_max = 0.8(m+1)/(eta0 dz)) against a domain too long to reach."""
    steps = 9000
    short = wl.c2_epstein(nz=3000, steps=steps, nfreq=4)
    short.wp2[:] = 0.0
    short.src_cell, short.probes = 1500, [600, 2400]
    off = steps + 50
    long = wl.c2_epstein(nz=3000 + 2 * off, steps=steps, nfreq=4)
    long.wp2[:] = 0.0
    long.nu = np.concatenate([np.full(off, short.nu[0]), short.nu, np.full(off, short.nu[-1])])
    long.src_cell, long.probes = 1500 + off, [600 + off, 2400 + off]
    _, s1 = oracle.run1d(short, series=True)
    _, s2 = oracle.run1d(long, series=True)
    peak = np.abs(s2).max()
    assert peak > 0.1
    assert np.abs(s1 - s2).max() <= 1e-4 * peak


def test_normalised_restatement_agrees_to_fp64_noise_floor():
    """P11: an independent NumPy restatement in normalised variables (the CUDA path's form)."""
    s = wl.c1_plain_slab(steps=3000)
    st, _ = oracle.run1d(s)
    E, H, J, X = an.normalized_run(s, s.steps)
    assert np.abs(E - st.E).max() <= 1e-13 * np.abs(st.E).max()
    assert np.abs(H - st.H).max() <= 1e-13 * np.abs(st.H).max()
    assert np.abs(J - st.J).max() <= 1e-13 * np.abs(st.J).max()
    assert np.abs(X - st.X).max() <= 1e-13 * np.abs(st.X).max()


def test_openmp_build_is_bitwise_equal_to_serial_build():
    s = wl.c2_epstein(nz=20000, steps=300, nfreq=8)
    a, sa = oracle.run1d(s, series=True)
    b, sb = oracle.run1d(s, series=True, omp=True)
    for f in ("E", "H", "J", "psiE", "psiH", "X"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert np.array_equal(sa, sb)


def test_resume_from_state_is_bitwise_equal_to_uninterrupted_run():
    s = wl.c2_epstein(nz=5000, steps=700, nfreq=8)
    s.probes = [2032, 4000]
    a, _ = oracle.run1d(s)
    b, _ = oracle.run1d(s, steps=300)
    b, _ = oracle.run1d(s, steps=400, state=b)
    for f in ("E", "H", "J", "psiE", "psiH", "X"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("mutant", [1, 2, 3, 4])
def test_pins_reject_planted_mistakes(mutant, c1_exact):
    """Each planted oracle mistake (printed Eq. 13, swapped Eq. 11 index, DFT sign, Mur sign)
    breaks the finite-lattice pin that the correct oracle passes at 1e-7 above 35 GHz."""
    Rd, Td = c1_exact
    R, T = _rt(wl.c1_plain_slab(steps=16000), mutant=mutant)
    hi = slice(70, None)
    err = max(np.abs(R - Rd)[hi].max(), np.abs(T - Td)[hi].max())
    assert err > 1e-5, err
