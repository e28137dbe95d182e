"""GPU parity of the 3D Yee RKETD step against the 3D oracle (and, where the problem reduces
to it, the 1D oracle). FP64: every field within 1e-11 of its group's peak; FP32: within
2e-4 of the peak (single-precision rounding over a few hundred steps)."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GROUPS = {"E": ("Ex", "Ey", "Ez"), "H": ("Hx", "Hy", "Hz"), "J": ("Jx", "Jy", "Jz")}
TOL = {"f64": 1e-11, "f32": 2e-4}


def _compare(ctx, st, prob, prec, spectra=True):
    worst = {}
    for grp, names in GROUPS.items():
        ref = {n: st.field(n, prob) for n in names}
        peak = max(np.abs(r).max() for r in ref.values())
        if peak == 0:
            for n in names:
                assert not np.any(ctx.field(n)), n
            continue
        for n in names:
            err = np.abs(ctx.field(n) - ref[n]).max() / peak
            worst[n] = err
            assert err <= TOL[prec], (n, err)
    if spectra and len(prob.probes):
        X = ctx.spectra()
        scale = np.abs(st.X).max()
        assert scale > 0
        err = np.abs(X - st.X).max() / scale
        worst["X"] = err
        assert err <= TOL[prec], ("X", err)
    return worst


def _sphere(n=37, steps=260):
    p = wl.sphere_problem(n=n, steps=steps, radius=5.0, npml=6, nfreq=8)
    p.box = (12, 24, 12, 24, 12, 24)
    return p


def _ragged():
    """Odd sizes on every axis (x not a multiple of the 32-wide tile, y not of 8), an
    off-centre sphere cut by the box, CPML of 5 cells, probes in both regions."""
    nx, ny, nz = 37, 29, 45
    d = 100e-6
    dt = wl.dt_for_courant(d, 0.5)
    m1 = wl.sphere_materials(nx, ny, nz, (17.3, 12.6, 23.9), 6.2, 1)
    m2 = wl.sphere_materials(nx, ny, nz, (24.0, 19.0, 30.0), 3.1, 2)
    assert not np.any((m1 != 0) & (m2 != 0))  # disjoint spheres: every 2-bit index stays 0, 1 or 2
    mat = m1 | m2
    freqs = 100e9 * np.arange(1, 9, dtype=float) / 8
    return wl.Grid3D(nx, ny, nz, d, dt, mat, np.array([0.0, (2 * math.pi * 40e9) ** 2, (2 * math.pi * 25e9) ** 2]),
                     np.array([0.0, 2e10, 7e10]), False, 5, True, (9, 27, 8, 21, 10, 35), -1, 15 * dt, 75 * dt,
                     [(17, 12, 7), (20, 14, 38), (18, 13, 22)], freqs, 230)


def _ragged16():
    """As _ragged with nx = 48, which the staged form takes (x a multiple of 16, not of the
    32-wide tile), the sphere cut by the box and the CPML near the x faces."""
    p = _ragged()
    nx, ny, nz = 48, p.ny, p.nz
    m1 = wl.sphere_materials(nx, ny, nz, (21.3, 12.6, 23.9), 6.2, 1)
    m2 = wl.sphere_materials(nx, ny, nz, (33.0, 19.0, 30.0), 3.1, 2)
    assert not np.any((m1 != 0) & (m2 != 0))
    p.nx, p.mat = nx, m1 | m2
    p.box = (9, 38, 8, 21, 10, 35)
    p.probes = [(21, 12, 7), (40, 14, 38), (18, 13, 22), (31, 20, 30)]
    return p


def _lean():
    """A grid whose middle tiles are clear of the CPML and of the TF/SF faces, so that the
    staged form takes its lean path there, with plasma of both materials inside them."""
    nx, ny, nz = 96, 40, 40
    d = 100e-6
    dt = wl.dt_for_courant(d, 0.5)
    m1 = wl.sphere_materials(nx, ny, nz, (47.6, 20.3, 19.8), 8.3, 1)
    m2 = wl.sphere_materials(nx, ny, nz, (70.2, 13.9, 26.1), 4.2, 2)
    assert not np.any((m1 != 0) & (m2 != 0))
    freqs = 100e9 * np.arange(1, 9, dtype=float) / 8
    return wl.Grid3D(nx, ny, nz, d, dt, m1 | m2, np.array([0.0, (2 * math.pi * 40e9) ** 2, (2 * math.pi * 25e9) ** 2]),
                     np.array([0.0, 2e10, 7e10]), False, 4, True, (8, 87, 6, 33, 7, 32), -1, 15 * dt, 75 * dt,
                     [(48, 20, 5), (60, 25, 36), (50, 18, 20)], freqs, 200)


def _faces():
    """The lean grid with the TF/SF box's x face (i = 40) and y face (Hz at j = 16) crossing
    tiles that are clear of the CPML, so those tiles take the faces-only boundary path."""
    p = _lean()
    p.box = (40, 87, 17, 33, 7, 32)
    return p


def _wide3():
    """The lean recipe on a grid 160 cells wide: three neighbouring interior tiles per row, with
    plasma across the boundary between the first two and a probe in the middle z range."""
    nx, ny, nz = 160, 40, 40
    d = 100e-6
    dt = wl.dt_for_courant(d, 0.5)
    m1 = wl.sphere_materials(nx, ny, nz, (63.4, 20.3, 19.8), 8.3, 1)
    m2 = wl.sphere_materials(nx, ny, nz, (104.2, 13.9, 26.1), 4.2, 2)
    assert not np.any((m1 != 0) & (m2 != 0))
    freqs = 100e9 * np.arange(1, 9, dtype=float) / 8
    return wl.Grid3D(nx, ny, nz, d, dt, m1 | m2, np.array([0.0, (2 * math.pi * 40e9) ** 2, (2 * math.pi * 25e9) ** 2]),
                     np.array([0.0, 2e10, 7e10]), False, 4, True, (8, 151, 6, 33, 7, 32), -1, 15 * dt, 75 * dt,
                     [(48, 20, 5), (66, 20, 20), (100, 18, 24)], freqs, 200)


GRIDS3 = {"ragged16": _ragged16, "lean": _lean, "faces": _faces, "wide3": _wide3}


@pytest.mark.parametrize("grid", ["ragged16", "lean", "faces", "wide3"])
@pytest.mark.parametrize("k_chunk", [0, 7, 45])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_staged_form_matches_the_3d_oracle(prec, k_chunk, grid):
    p = GRIDS3[grid]()
    st, _ = oracle.run3d(p)
    with rk.Context3D(p, prec, variant="staged", k_chunk=k_chunk) as ctx:
        ctx.step(100)
        ctx.step(p.steps - 100)
        worst = _compare(ctx, st, p, prec)
    print(prec, "staged", k_chunk, {k: f"{v:.2e}" for k, v in worst.items()})


@pytest.mark.parametrize("grid", ["ragged16", "lean", "faces", "wide3"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_staged_form_agrees_bitwise_with_the_plain_form(prec, grid):
    p = GRIDS3[grid]()
    out = []
    for variant, kc in (("plain", 0), ("staged", 0), ("staged", 3), ("auto", 0)):
        with rk.Context3D(p, prec, variant=variant, k_chunk=kc) as ctx:
            ctx.step(151)
            out.append(([ctx.field(n) for n in rk.FIELDS_3D], ctx.spectra()))
    for f, X in out[1:]:
        assert all(np.array_equal(u, v) for u, v in zip(out[0][0], f))
        assert np.array_equal(out[0][1], X)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_staged_form_with_a_sheet_source_matches_the_3d_oracle(prec):
    """The sheet plane crosses interior and boundary tiles; no TF/SF box."""
    p = _lean()
    p.tfsf = False
    p.sheet_k = 12
    p.steps = 150
    st, _ = oracle.run3d(p)
    with rk.Context3D(p, prec, variant="staged", k_chunk=9) as ctx:
        ctx.step(p.steps)
        worst = _compare(ctx, st, p, prec)
    print(prec, "staged sheet", {k: f"{v:.2e}" for k, v in worst.items()})


def test_staged_form_is_refused_where_it_does_not_apply():
    p = _ragged()  # nx = 37
    with pytest.raises(rk.RketdError) as ei:
        rk.Context3D(p, "f32", variant="staged")
    assert ei.value.status == 6


@pytest.mark.parametrize("variant", ["plain", "fused"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sphere_tfsf_cpml_matches_the_3d_oracle(prec, variant):
    p = _sphere()
    st, _ = oracle.run3d(p)
    with rk.Context3D(p, prec, variant=variant) as ctx:
        ctx.step(p.steps)
        worst = _compare(ctx, st, p, prec)
    print(prec, variant, {k: f"{v:.2e}" for k, v in worst.items()})


@pytest.mark.parametrize("variant,k_chunk", [("plain", 0), ("fused", 0), ("fused", 7), ("fused", 1)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_grid_two_materials_matches_the_3d_oracle(prec, variant, k_chunk):
    p = _ragged()
    st, _ = oracle.run3d(p)
    with rk.Context3D(p, prec, variant=variant, k_chunk=k_chunk) as ctx:
        ctx.step(100)
        ctx.step(p.steps - 100)  # split calls: the DFT fold and the step index carry over
        worst = _compare(ctx, st, p, prec)
    print(prec, variant, k_chunk, {k: f"{v:.2e}" for k, v in worst.items()})


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_plain_and_fused_forms_and_chunkings_agree_bitwise(prec):
    """The two forms run the same operations in the same order on every value; the chunk of
    z planes per block changes only which thread does them."""
    p = _ragged()
    p.probes = [(17, 12, 7), (20, 14, 38), (18, 13, 22), (18, 13, 23)]
    out = []
    for variant, kc in (("plain", 0), ("fused", 0), ("fused", 5), ("fused", 45)):
        with rk.Context3D(p, prec, variant=variant, k_chunk=kc) as ctx:
            ctx.step(177)
            out.append(([ctx.field(n) for n in rk.FIELDS_3D], ctx.spectra()))
    for f, X in out[1:]:
        assert all(np.array_equal(u, v) for u, v in zip(out[0][0], f))
        assert np.array_equal(out[0][1], X)


def test_periodic_layered_slab_reduces_to_the_1d_oracle():
    nx, ny, nz, steps = 4, 8, 260, 700
    d = 75e-6
    dt = wl.dt_for_courant(d, 0.5)
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[140:170] = 1 | (1 << 2) | (1 << 4)
    freqs = 0.5e9 * np.arange(1, 41, dtype=float)
    p = wl.Grid3D(nx, ny, nz, d, dt, mat.ravel(), np.array([0.0, (2 * math.pi * 28.7e9) ** 2]),
                  np.array([0.0, 2e10]), True, 16, False, (0, 0, 0, 0, 0, 0), 60, 15 * dt, 75 * dt,
                  [(1, 2, 40), (3, 5, 220)], freqs, steps)
    s1 = wl.Slab1D(nz, d, dt, np.zeros(nz), np.zeros(nz), 60, 15 * dt, 75 * dt, [40, 220], freqs, "cpml", 16, steps)
    s1.wp2[140:170] = p.mat_wp2[1]
    s1.nu[140:170] = p.mat_nu[1]
    st1, _ = oracle.run1d(s1)
    with rk.Context3D(p, "f64", k_chunk=11) as ctx:
        ctx.step(steps)
        Ex, Hy, Jx = ctx.field("Ex"), ctx.field("Hy"), ctx.field("Jx")
        X = ctx.spectra()
        for n in ("Ey", "Ez", "Hx", "Hz", "Jy", "Jz"):
            assert not np.any(ctx.field(n)), n
    pe, ph = np.abs(st1.E).max(), np.abs(st1.H).max()
    for j in range(ny):
        for i in range(nx):
            assert np.abs(Ex[:, j, i] - st1.E).max() <= 1e-11 * pe
            assert np.abs(Hy[:-1, j, i] - st1.H).max() <= 1e-11 * ph
            assert np.abs(Jx[:, j, i] - st1.J).max() <= 1e-11 * np.abs(st1.J).max()
    assert np.abs(X - st1.X).max() <= 1e-11 * np.abs(st1.X).max()


@pytest.mark.parametrize("variant", ["plain", "fused"])
def test_sheet_source_on_a_closed_grid_matches_the_3d_oracle(variant):
    """CPML on all faces with the soft sheet source: the sheet covers the whole plane, the
    PEC wall cells included, as in the oracle."""
    p = _sphere(n=33, steps=150)
    p.tfsf = False
    p.sheet_k = 9
    st, _ = oracle.run3d(p)
    with rk.Context3D(p, "f64", variant=variant) as ctx:
        ctx.step(p.steps)
        _compare(ctx, st, p, "f64")


def test_reset_reproduces_the_first_run_bitwise():
    p = _ragged()
    with rk.Context3D(p, "f32") as ctx:
        ctx.step(120)
        a = [ctx.field(n) for n in ("Ex", "Hy", "Jz")]
        Xa = ctx.spectra()
        ctx.reset()
        ctx.step(120)
        b = [ctx.field(n) for n in ("Ex", "Hy", "Jz")]
        assert all(np.array_equal(u, v) for u, v in zip(a, b))
        assert np.array_equal(Xa, ctx.spectra())
        assert ctx.launches >= 240  # one fused launch per step


def test_full_size_sphere_grid_total_field_is_the_incident_wave():
    """512^3 FP32 as in the benchmark, 260 steps: the pulse is inside the TF/SF box but has
    not reached the sphere (k >= 136), so the total field in the box equals the incident line,
    which is the 1D oracle on a vacuum line of the same length, and the scattered-field region
    holds only rounding. Checks every box face and the indexing at full size."""
    p = wl.sphere_problem(n=512, steps=260)
    steps = 260
    line = wl.Slab1D(p.inc_len, p.d, p.dt, np.zeros(p.inc_len), np.zeros(p.inc_len), p.inc_src, p.src_tau,
                     p.src_t0, [p.inc_off + 30], np.array([1e9]), "mur", 0, steps)
    st1, _ = oracle.run1d(line)
    inc = st1.E[np.arange(p.nz) + p.inc_off]
    peak = np.abs(inc).max()
    i0, i1, j0, j1, k0, k1 = p.box
    assert np.abs(inc[k0 + 20:k1 + 1]).max() > 0.5 * peak  # the pulse is well inside the box
    assert np.abs(inc[136:]).max() < 1e-6 * peak  # and has not reached the sphere
    with rk.Context3D(p, "f32") as ctx:
        ctx.step(steps)
        Ex = ctx.field("Ex")
        inside = Ex[k0:k1 + 1, j0:j1 + 1, i0:i1]
        assert np.abs(inside - inc[k0:k1 + 1, None, None]).max() <= 2e-4 * peak
        Ex[k0:k1 + 1, j0:j1 + 1, i0:i1] = 0.0
        assert np.abs(Ex).max() <= 2e-5 * peak
        del Ex, inside
        for n in ("Ey", "Ez"):
            assert np.abs(ctx.field(n)).max() <= 2e-5 * peak, n


def test_grid_without_probes_steps_and_returns_fields():
    """No probes (no DFT buffers): the step, the fields and the (empty) spectra still work, and the
    fields equal those of the same run with probes."""
    p = _lean()
    p.steps = 60
    with rk.Context3D(p, "f32") as ref:
        ref.step(p.steps)
        ex_ref = ref.field("Ex")
    q = _lean()
    q.probes = []
    with rk.Context3D(q, "f32") as ctx:
        ctx.step(0)
        ctx.step(p.steps)
        assert np.array_equal(ctx.field("Ex"), ex_ref)
        assert ctx.spectra().shape == (0, len(q.freq_hz))


@pytest.fixture(scope="module")
def sphere128():
    """The benchmark's sphere recipe on a 128^3 grid (radius 30, TF/SF box 20..107, 16-cell CPML on
    every face), 300 steps: the pulse crosses the whole sphere."""
    p = wl.sphere_problem(n=128, steps=300, nfreq=16)
    st, _ = oracle.run3d(p)
    return p, st


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_staged_form_matches_the_3d_oracle_on_the_128_cube_sphere(sphere128, prec):
    p, st = sphere128
    with rk.Context3D(p, prec) as ctx:
        ctx.step(p.steps)
        worst = _compare(ctx, st, p, prec)
    print(prec, "128^3", {k: f"{v:.2e}" for k, v in worst.items()})
