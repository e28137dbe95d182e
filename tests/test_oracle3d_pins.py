"""Pins of the 3D oracle (CPU only): exact reduction to the 1D oracle, and the total-field /
scattered-field box reproducing the incident plane wave inside and nothing outside."""
import math

import numpy as np

import oracle
from paper_1709_00821_gb300 import workloads as wl


def _layered(nx=4, ny=4, nz=260, steps=700):
    """Periodic x, y; CPML along z; sheet source on Ex at k = 60; plasma on 140 <= k < 170."""
    d = 75e-6
    dt = wl.dt_for_courant(d, 0.5)
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[140:170] = 1 | (1 << 2) | (1 << 4)  # Ex, Ey and Ez of the layer cells in material 1
    prob = wl.Grid3D(nx, ny, nz, d, dt, mat.ravel(), np.array([0.0, (2 * math.pi * 28.7e9) ** 2]),
                     np.array([0.0, 2e10]), True, 16, False, (0, 0, 0, 0, 0, 0), 60, 15 * dt, 75 * dt,
                     [(1, 2, 40), (2, 1, 220)], 0.5e9 * np.arange(1, 41, dtype=float), steps)
    s1 = wl.Slab1D(nz, d, dt, np.zeros(nz), np.zeros(nz), 60, 15 * dt, 75 * dt,
                   [40, 220], prob.freq_hz, "cpml", 16, steps)
    s1.wp2[140:170] = prob.mat_wp2[1]
    s1.nu[140:170] = prob.mat_nu[1]
    return prob, s1


def test_periodic_layered_3d_reduces_bitwise_to_the_1d_oracle():
    prob, s1 = _layered()
    st3, _ = oracle.run3d(prob)
    st1, _ = oracle.run1d(s1)
    Ex = st3.field("Ex", prob)
    Hy = st3.field("Hy", prob)
    Jx = st3.field("Jx", prob)
    for j in range(prob.ny):
        for i in range(prob.nx):
            assert np.array_equal(Ex[:, j, i], st1.E)
            assert np.array_equal(Hy[:-1, j, i], st1.H)
            assert np.array_equal(Jx[:, j, i], st1.J)
    for name in ("Ey", "Ez", "Hx", "Hz", "Jy", "Jz"):
        assert not np.any(st3.field(name, prob)), name
    assert np.array_equal(st3.X, st1.X)


def _vacuum_box(n=36, steps=125, npml=6):
    p = wl.sphere_problem(n=n, steps=steps, radius=0.0, npml=npml, nfreq=8)
    p.mat = np.zeros_like(p.mat)
    lo, hi = 11, n - 12
    p.box = (lo, hi, lo, hi, lo, hi)
    return p


def test_tfsf_box_in_vacuum_holds_the_incident_wave_and_leaks_nothing():
    p = _vacuum_box()
    st, _ = oracle.run3d(p)
    Ex = st.field("Ex", p)
    i0, i1, j0, j1, k0, k1 = p.box
    inc = st.inc[0][np.arange(p.nz) + p.inc_off]
    peak = np.abs(inc).max()
    assert peak > 0.05  # the pulse is inside the box at the end of the run
    # total field inside the box = incident plane wave (Ex components inside: i0 <= i <= i1-1)
    inside = Ex[k0:k1 + 1, j0:j1 + 1, i0:i1]
    assert np.abs(inside - inc[k0:k1 + 1, None, None]).max() <= 1e-12 * peak
    # scattered field outside the box: nothing
    mask = np.ones_like(Ex, bool)
    mask[k0:k1 + 1, j0:j1 + 1, i0:i1] = False
    assert np.abs(Ex[mask]).max() <= 1e-12 * peak
    for name in ("Ey", "Ez", "Hx", "Hz"):
        assert np.abs(st.field(name, p)).max() <= 1e-12 * peak, name


def test_plasma_sphere_scatters_into_the_scattered_field_region():
    # odd grid: every ingredient (CPML depths, box, sphere) is mirror-symmetric about node 18
    p = wl.sphere_problem(n=37, steps=260, radius=5.0, npml=6, nfreq=8)
    p.box = (12, 24, 12, 24, 12, 24)
    st, ser = oracle.run3d(p, series=True)
    assert np.abs(ser[0]).max() > 1e-6  # backscatter reaches the probe before the box
    # symmetry of an x-polarised wave along z on a centred sphere: Ex is even in y about the centre
    Ex = st.field("Ex", p)
    c = p.ny // 2
    assert np.abs(Ex[:, c + 3, :] - Ex[:, c - 3, :]).max() <= 1e-12 * np.abs(Ex).max()
