"""Pins of the oracle adjoint (CPU only): derivatives of phi1/phi2 against 40-digit
differentiation, the transposed step against the forward step (dot-product identity), and
loss gradients against central finite differences of the forward oracle."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import workloads as wl


def test_phi_derivatives_match_40_digit_differentiation():
    mp.mp.dps = 40
    f1 = lambda x: (1 - mp.e ** (-x)) / x
    f2 = lambda x: (mp.e ** (-x) - 1 + x) / x ** 2
    for x in [1e-9, 2.5e-3, 0.05, 0.5, 0.999, 1.0, 1.5, 4.0, 40.0]:
        d1 = float(mp.diff(f1, mp.mpf(x)))
        d2 = float(mp.diff(f2, mp.mpf(x)))
        assert abs(oracle.dphi1(x) - d1) <= 1e-14 * abs(d1) + 1e-300, x
        assert abs(oracle.dphi2(x) - d2) <= 1e-14 * abs(d2) + 1e-300, x


def _random_slab(nz=64, seed=3):
    s = wl.c1_plain_slab(nz=nz, steps=1)
    u = wl.uniform01(seed, 2 * nz)
    s.wp2 = (2 * math.pi * 50e9 * u[:nz]) ** 2
    s.nu = 5e10 * u[nz:]
    s.src_amp = 0.0
    s.src_cell, s.probes = nz // 3, [2, nz - 3]
    return s


def test_transposed_step_satisfies_the_dot_product_identity():
    """<A x, y> = <x, A^T y> for one step (Eqs. 14, 13, 11, Mur ends), random x and y."""
    s = _random_slab()
    nz = s.nz
    g = wl.normal(21, 6 * nz)
    x = oracle.State1D(s)
    x.E[:], x.H[:], x.J[:] = g[:nz], g[nz:2 * nz - 1], g[2 * nz:3 * nz]
    ax, _ = oracle.run1d(s, steps=1, state=x.copy())
    yE, yH, yJ = g[3 * nz:4 * nz], g[4 * nz:5 * nz - 1], g[5 * nz:6 * nz]
    lE, lH, lJ = oracle.adjoint_step(s, yE, yH, yJ)
    lhs = ax.E @ yE + ax.H @ yH + ax.J @ yJ
    rhs = x.E @ lE + x.H @ lH + x.J @ lJ
    scale = np.abs(ax.E * yE).sum() + np.abs(ax.H * yH).sum() + np.abs(ax.J * yJ).sum()
    assert abs(lhs - rhs) <= 1e-14 * scale


def _problem(nz=700, steps=1600):
    """Smooth random plasma profile on cells [300, 400), reflection probe at 150."""
    s = wl.c1_plain_slab(nz=nz, steps=steps)
    s.src_cell, s.probes = 100, [150, 600]
    s.freq_hz = np.linspace(5e9, 100e9, 24)
    base = wl.c4_profile(0, nz=nz, region=(300, 400), steps=steps)
    s.wp2, s.nu = base.wp2.copy(), base.nu.copy()
    tgt = wl.c4_profile(1000, nz=nz, region=(300, 400), steps=steps)
    return s, tgt


def _loss(s, X_inc, R_t):
    st, _ = oracle.run1d(s)
    return oracle.reflection_loss(st.X, X_inc, R_t)


@pytest.fixture(scope="module")
def adj_case():
    s, tgt = _problem()
    inc, _ = oracle.run1d(s.vacuum())
    t_tot, _ = oracle.run1d(tgt_from(s, tgt))
    R_t = np.abs((t_tot.X[0] - inc.X[0]) / inc.X[0])
    L, gX = _loss(s, inc.X, R_t)
    gw, gn = oracle.adjoint(s, gX)
    return s, inc, R_t, L, gw, gn


def tgt_from(s, tgt):
    t = s.vacuum()
    t.wp2, t.nu = tgt.wp2.copy(), tgt.nu.copy()
    return t


def test_adjoint_gradient_matches_central_differences_along_a_direction(adj_case):
    s, inc, R_t, L, gw, gn = adj_case
    assert L > 0
    d = wl.normal(77, 2 * s.nz)
    mask = (s.wp2 > 0).astype(float)
    dw = d[:s.nz] * mask * s.wp2.max()
    dn = d[s.nz:] * mask * 1e10
    h = 1e-5
    sp, sm = s.vacuum(), s.vacuum()
    sp.wp2, sp.nu = s.wp2 + h * dw, s.nu + h * dn
    sm.wp2, sm.nu = s.wp2 - h * dw, s.nu - h * dn
    fd = (_loss(sp, inc.X, R_t)[0] - _loss(sm, inc.X, R_t)[0]) / (2 * h)
    ad = gw @ dw + gn @ dn
    assert abs(ad - fd) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("cell", [301, 317, 333, 350, 366, 382, 398, 360])
def test_adjoint_gradient_matches_central_differences_at_single_cells(adj_case, cell):
    s, inc, R_t, L, gw, gn = adj_case
    region = s.wp2 > 0
    for arr, g, h in (("wp2", gw, 1e-6 * s.wp2.max()), ("nu", gn, 1e-4 * s.nu[region].max())):
        sp, sm = s.vacuum(), s.vacuum()
        sp.wp2, sp.nu, sm.wp2, sm.nu = s.wp2.copy(), s.nu.copy(), s.wp2.copy(), s.nu.copy()
        getattr(sp, arr)[cell] += h
        getattr(sm, arr)[cell] -= h
        fd = (_loss(sp, inc.X, R_t)[0] - _loss(sm, inc.X, R_t)[0]) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(g[region]).max())
        assert abs(g[cell] - fd) <= 1e-5 * scale, (arr, cell, g[cell], fd)


def test_gradient_vanishes_outside_the_plasma(adj_case):
    s, inc, R_t, L, gw, gn = adj_case
    # nu enters only through J, which stays zero where wp2 = 0
    assert np.all(gn[s.wp2 == 0] == 0)
    assert np.abs(gw[:100]).max() < np.abs(gw).max()
