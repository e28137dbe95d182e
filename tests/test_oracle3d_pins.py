"""Pins of the 3D oracle (CPU only), none of which uses the oracle to check itself:

* exact reduction to the 1D oracle along z, for Ex/Hy (sheet source) and Ey/Hx (initial profile);
* a single transverse Fourier mode obeys the lattice recurrence derived from Eqs. 11, 12, 14 and keeps
  its shape (every bulk x and y difference term, in vacuum and in plasma);
* a cyclic rotation of the cube maps the x- and y-face CPML onto the z-face CPML bit for bit;
* the x/y-face CPML reflects below 1e-3 of the scattered field (against a domain whose faces are
  out of reach);
* the total-field/scattered-field box reproduces the incident plane wave inside and nothing outside;
* planted mistakes in the transverse terms and the x/y-face CPML fail these pins.
"""
import math

import analytic
import numpy as np
import pytest

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


# ---------------------------------------------------------------------------------------------
# Transverse operators and the x/y-face CPML (Eqs. 1-3 in full curl form).
# ---------------------------------------------------------------------------------------------

def _grid(nx, ny, nz, periodic, npml, mat, wp2=0.0, nu=0.0, d=75e-6, steps=1):
    dt = wl.dt_for_courant(d, 0.5)
    return wl.Grid3D(nx, ny, nz, d, dt, np.asarray(mat, np.uint8).ravel(), np.array([0.0, wp2]),
                     np.array([0.0, nu]), periodic, npml, False, (0,) * 6, -1, 15 * dt, 75 * dt, [],
                     np.array([1e9]), steps)


def _mode_recurrence(S, mu, w, x):
    """Coefficients c0..c3 of the recurrence every field sample of one spatial Fourier mode obeys.

    With the mode's discrete Laplacian eigenvalue -mu/d^2 (mu = 4 sin^2(kx d/2) + 4 sin^2(ky d/2)),
    eliminating H from Eqs. 12 and 14 gives E^{n+1} - 2E^n + E^{n-1} = -S^2 mu E^n
    - (J~^{n+1} - J~^{n-1})/2 (J~ = dt J/eps0), and Eq. 11 gives J~ = (w phi2 z + w(phi1 - phi2))/(z - a) E
    in z-transform. Clearing denominators, every sample obeys the cubic
    (z^2 - A z + 1)(z - a) + (z^2 - 1)(p z + q)/2 = 0, A = 2 - S^2 mu, p = w phi2, q = w (phi1 - phi2).
    In vacuum (w = 0) it reduces to (z - a)(z^2 - A z + 1): cos(theta) = 1 - S^2 mu/2, i.e.
    sin^2(theta/2) = S^2 (sin^2(kx d/2) + sin^2(ky d/2)), the 2D Yee dispersion relation.
    """
    p1, p2 = analytic.phi_mp(x)
    a = math.exp(-x)
    p, q = w * p2, w * (p1 - p2)
    A = 2.0 - S * S * mu
    return np.array([-a - q / 2, 1 + a * A - p / 2, -(A + a) + q / 2, 1 + p / 2])


def _run_mode(kind, plasma, steps=60, mutant=0):
    """One Fourier mode (kx, ky) = 2 pi (2/16, 1/12) on a periodic 16 x 12 grid, uniform in z.

    TM (Ez, Hx, Hy): Ez is normal to the PEC z walls, so the mode is exact on every plane and the
    z-CPML is never driven. TE (Hz, Ex, Ey): the walls' influence spreads one plane per step, so
    the middle plane of a grid 2 steps + 10 planes deep evolves as on an unbounded grid.
    Returns (time series of the mode's component on the middle plane [n, j, i], recurrence coeffs).
    """
    nx, ny = 16, 12
    nz = 2 * steps + 10 if kind == "TE" else 12
    wp2, nu = ((2 * math.pi * 30e9) ** 2, 2e10) if plasma else (0.0, 0.0)
    mat = np.full((nz, ny, nx), 1 | (1 << 2) | (1 << 4) if plasma else 0, np.uint8)
    p = _grid(nx, ny, nz, True, 3, mat, wp2, nu)
    st = oracle.State3D(p)
    kx, ky = 2 * math.pi * 2 / nx, 2 * math.pi * 1 / ny
    i, j = np.arange(nx), np.arange(ny)
    F = st.fields.reshape(9, nz, ny, nx)
    if kind == "TM":  # Ez at (i, j, k + 1/2)
        F[2, :nz - 1] = np.cos(kx * i[None, :] + ky * j[:, None])[None]
        comp = 2
    else:  # Hz at (i + 1/2, j + 1/2, k)
        F[5] = np.cos(kx * (i[None, :] + 0.5) + ky * (j[:, None] + 0.5))[None]
        comp = 5
    kc = nz // 2
    ser = []
    for _ in range(steps):
        ser.append(st.fields.reshape(9, nz, ny, nx)[comp, kc].copy())
        st, _ = oracle.run3d(p, steps=1, state=st, mutant=mutant)
    S = analytic.courant(p.d, p.dt)
    mu = 4 * (math.sin(kx / 2) ** 2 + math.sin(ky / 2) ** 2)
    return np.array(ser), _mode_recurrence(S, mu, wp2 * p.dt ** 2, nu * p.dt)


def _mode_residuals(ser, c):
    res = c[0] * ser[:-3] + c[1] * ser[1:-2] + c[2] * ser[2:-1] + c[3] * ser[3:]
    rec = np.abs(res).max() / (np.abs(ser).max() * np.abs(c).sum())
    pat = ser[0]
    amp = (ser * pat).sum(axis=(1, 2)) / (pat * pat).sum()
    shape = np.abs(ser - amp[:, None, None] * pat).max() / np.abs(ser).max()
    return rec, shape


@pytest.mark.parametrize("plasma", [False, True])
@pytest.mark.parametrize("kind", ["TM", "TE"])
def test_transverse_mode_obeys_the_exact_lattice_recurrence(kind, plasma):
    """Pins every x and y difference term of the bulk curl (TM: Hx's dEz/dy, Hy's dEz/dx and
    Ez's two; TE: Hz's two, Ex's dHz/dy and Ey's dHz/dx) and their plasma coupling: a single
    Fourier mode keeps its spatial shape to round-off, and its samples obey the lattice
    recurrence of _mode_recurrence to round-off (3e-16 measured)."""
    ser, c = _run_mode(kind, plasma)
    rec, shape = _mode_residuals(ser, c)
    assert np.abs(ser).max() > 0.5
    assert rec <= 1e-14, rec
    assert shape <= 1e-13, shape


def test_y_polarised_layered_3d_reduces_bitwise_to_the_1d_oracle():
    """Ey/Hx along z (the z terms of the Ey and Hx updates and their z-CPML memories) on a
    periodic grid, from a Gaussian Ey profile: Ey, -Hx, Jy equal the 1D oracle's E, H, J started
    from the same profile, bit for bit (dHx/dz = -dH/dz exactly, with kappa = 1)."""
    nz, steps = 200, 300
    mat = np.zeros((nz, 4, 4), np.uint8)
    mat[120:150] = 1 << 2  # Ey of the layer cells in plasma
    p = _grid(4, 4, nz, True, 12, mat, (2 * math.pi * 28.7e9) ** 2, 2e10, steps=steps)
    k = np.arange(nz)
    E0 = np.exp(-((k - 70) / 8.0) ** 2)
    E0[0] = E0[-1] = 0.0
    st = oracle.State3D(p)
    st.fields.reshape(9, nz, 4, 4)[1] = E0[:, None, None]
    st, _ = oracle.run3d(p, state=st)
    s1 = wl.Slab1D(nz, p.d, p.dt, np.zeros(nz), np.zeros(nz), 5, p.src_tau, p.src_t0, [], np.array([1e9]), "cpml",
                   12, steps, 0.0)
    s1.wp2[120:150] = p.mat_wp2[1]
    s1.nu[120:150] = p.mat_nu[1]
    st1 = oracle.State1D(s1)
    st1.E[:] = E0
    st1, _ = oracle.run1d(s1, state=st1)
    assert np.abs(st1.J).max() > 1e-3 and np.abs(st1.psiE).max() > 0
    F = st.fields.reshape(9, nz, 4, 4)
    for j in range(4):
        for i in range(4):
            assert np.array_equal(F[1][:, j, i], st1.E)
            assert np.array_equal(-F[3][:-1, j, i], st1.H)
            assert np.array_equal(F[7][:, j, i], st1.J)
    for q in (0, 2, 4, 5, 6, 8):
        assert not np.any(F[q]), q


def _rotate(F):
    """Cyclic rotation of a cube's fields [9][n][n][n] ([k][j][i]): old x -> new y, old y -> new z,
    old z -> new x, i.e. new (Ey, Ez, Ex)[j, i, k] = old (Ex, Ey, Ez)[k, j, i], and the same for H
    and J. It maps the Yee lattice onto itself (Ex at (i+1/2, j, k) lands on Ey at (k, i+1/2, j))."""
    G = np.empty_like(F)
    for b in (0, 3, 6):
        G[b + 1] = F[b + 0].transpose(1, 2, 0)
        G[b + 2] = F[b + 1].transpose(1, 2, 0)
        G[b + 0] = F[b + 2].transpose(1, 2, 0)
    return G


def _rotation_pair(mutant=0, n=22, steps=40):
    d = 100e-6
    mat = wl.sphere_materials(n, n, n, (10.7, 10.7, 10.7), 5.3, 1)  # invariant under the rotation
    p = _grid(n, n, n, False, 5, np.zeros(1), (2 * math.pi * 40e9) ** 2, 2e10, d=d, steps=steps)
    p.mat = mat
    rng = np.random.default_rng(0x3D)
    F0 = rng.standard_normal((9, n, n, n))
    F0[3:6] /= 376.73
    F0[6:] *= 1e-3
    a = oracle.State3D(p)
    a.fields[:] = F0.reshape(9, -1)
    b = oracle.State3D(p)
    b.fields[:] = _rotate(F0).reshape(9, -1)
    a, _ = oracle.run3d(p, state=a, mutant=mutant)
    b, _ = oracle.run3d(p, state=b, mutant=mutant)
    return _rotate(a.fields.reshape(9, n, n, n)), b.fields.reshape(9, n, n, n), a


def test_cyclic_rotation_maps_the_x_and_y_face_cpml_onto_the_z_face_cpml():
    """On a cube with CPML on every face and a centred sphere, rotating a random initial state
    cyclically and running gives the rotated run bit for bit: the x- and y-face CPML memories
    (Ex/y, Ey/x, Ez/x, Ez/y, Hx/y, Hy/x, Hz/x, Hz/y) behave exactly as the z-face ones, which the
    two layered reductions pin against the 1D oracle."""
    ra, b, a = _rotation_pair()
    assert all(np.count_nonzero(a.psi[q]) > 1000 for q in range(12))
    assert np.array_equal(ra, b)


def _cpml_problem(margin, steps=120, npml=6, mutant=0):
    """32^3 sphere problem (radius 4.5, TF/SF box 10..21, pulse tau = 5 dt) with `margin` extra cells
    of vacuum on each x and y side; probes in the scattered-field region around the box."""
    n, m = 32, margin
    d = 100e-6
    dt = wl.dt_for_courant(d, 0.5)
    N = n + 2 * m
    mat = wl.sphere_materials(N, N, n, (16.0 + m, 16.0 + m, 16.0), 4.5, 1)
    c = 16 + m
    probes = [(c, c, 8), (8 + m, c, 16), (c, 8 + m, 16), (23 + m, 23 + m, 23), (c, c, 24), (8 + m, 8 + m, 8)]
    return wl.Grid3D(N, N, n, d, dt, mat, np.array([0.0, (2 * math.pi * 40e9) ** 2]), np.array([0.0, 2e10]), False,
                     npml, True, (10 + m, 21 + m, 10 + m, 21 + m, 10, 21), -1, 5 * dt, 25 * dt, probes,
                     np.array([1e9]), steps)


def _cpml_reflection(mutant=0, steps=120):
    a = _cpml_problem(0, steps)
    b = _cpml_problem(steps, steps)  # x/y faces beyond the domain of dependence (one cell per step)
    _, sa = oracle.run3d(a, series=True, mutant=mutant)
    _, sb = oracle.run3d(b, series=True)
    return [np.abs(sa[q] - sb[q]).max() / np.abs(sb[q]).max() for q in range(len(a.probes))]


@pytest.mark.slow
def test_x_and_y_face_cpml_reflect_below_1e_3_of_the_scattered_field():
    """The sphere's scattered field meets the x and y faces of a 32^3 grid (6-cell CPML) at every
    angle; the same problem with those faces 120 cells farther out (beyond anything 120 steps can
    reach) has no x/y-face reflection. The probe series of the two differ by the reflection only:
    at most 1e-3 of the scattered-field peak at each probe (2e-4 measured; a polynomial-graded PML
    of this depth reflects about e^{-1.6 N cos(theta)} in the continuum, 1e-4 at normal incidence,
    1e-2 at 60 degrees, and the lattice adds its own small reflection)."""
    errs = _cpml_reflection()
    assert max(errs) <= 1e-3, errs


@pytest.mark.parametrize("mutant", [5, 6, 7, 8])
def test_planted_mistakes_in_the_3d_transverse_operators_fail_a_pin(mutant):
    """5: Ey's x term with the wrong sign; 6: Hx's y difference taken along x; 7: Hy's x-face CPML
    graded at the E nodes; 8: Ex's y-face CPML memory driven with the wrong sign."""
    failed = []
    for kind in ("TM", "TE"):
        rec, shape = _mode_residuals(*_run_mode(kind, True, mutant=mutant))
        if rec > 1e-14 or shape > 1e-13:
            failed.append(kind)
    ra, b, _ = _rotation_pair(mutant)
    if not np.array_equal(ra, b):
        failed.append("rotation")
    assert failed, mutant
    if mutant in (7, 8):
        assert "rotation" in failed
    if mutant == 5:
        assert "TE" in failed
    if mutant == 6:
        assert "TM" in failed
