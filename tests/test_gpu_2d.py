"""GPU parity of the 2D TMz/TEz step against the 2D oracle (which the CPU tests pin to the 1D
oracle at normal incidence, to the exact lattice recurrence of a 2D Fourier mode, and to the lattice
response of a layer at oblique incidence). FP64: every component within 1e-12 of its group's scale
(E, H, J; the largest magnitude the group reached during the run, since rounding errors are set by
that and not by the decayed final field) and the spectra within 1e-12 of their peak; FP32: 2e-4 of
the same scales (single-precision rounding over a few thousand steps), and R/T of the oblique mode
within 1e-4 absolute of the FP64 oracle where the incident spectrum holds at least 10% of its peak."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-4}
GROUPS = {"tm": (("Ez",), ("Hx", "Hy"), ("Jz",)), "te": (("Ex", "Ey"), ("Hz",), ("Jx", "Jy"))}


def _ragged(pol, periodic=False, nx=37):
    """Odd sizes (nx = 37: the one-cell kernels; nx = 36: the four-cells-per-thread kernels), Mur (or
    periodic) x, three materials in blobs and a stripe, a random source profile, probes in both halves
    and on the source row."""
    ny = 53
    d = 300e-6
    dt = wl.dt_for_courant(d, 0.5)
    j, i = np.mgrid[0:ny, 0:nx]
    mat = np.zeros((ny, nx), np.uint8)
    mat[((i - 20.3) ** 2 + (j - 30.1) ** 2) < 40] = 1
    mat[((i - 9.5) ** 2 + (j - 40.2) ** 2) < 12] = 2
    mat[17:21, :] = np.where(mat[17:21, :] == 0, 3, mat[17:21, :])
    prof = 0.5 + wl.uniform01(0x2D, nx)
    return wl.Grid2D(nx, ny, d, dt, pol, periodic, mat.ravel(),
                     np.array([0.0, (2 * math.pi * 40e9) ** 2, (2 * math.pi * 25e9) ** 2, (2 * math.pi * 15e9) ** 2]),
                     np.array([0.0, 2e10, 7e10, 1e9]), 7, prof, 5 * dt, 25 * dt,
                     [(3, 10), (30, 45), (18, 7), (0, 26)], 100e9 * np.arange(1, 9, dtype=float) / 8, 450)


def _oracle_with_scales(p, chunk=25):
    """The oracle's final state and, per field group, the largest magnitude it held at any step
    boundary that is a multiple of chunk (and at the end)."""
    st, scale = None, {}
    done = 0
    while done < p.steps:
        n = min(chunk, p.steps - done)
        st, _ = oracle.run2d(p, steps=n, state=st)
        done += n
        for names in GROUPS[p.pol]:
            scale[names] = max(scale.get(names, 0.0), max(np.abs(st.field(x, p)).max() for x in names))
    return st, scale


def _oblique(pol):
    p = wl.slab_2d(64, 400, pol, mode=1, steps=3000)
    p.src_tau = 5 * p.dt
    p.src_t0 = 5 * p.src_tau
    return p


CASES = {"ragged": lambda pol: _ragged(pol), "ragged_periodic": lambda pol: _ragged(pol, True),
         "quad": lambda pol: _ragged(pol, nx=36), "quad_periodic": lambda pol: _ragged(pol, True, nx=36),
         "oblique": _oblique, "normal": lambda pol: wl.slab_2d(4, 400, pol, mode=0, steps=1500, d=75e-6)}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("pol", ["tm", "te"])
def test_2d_step_matches_the_2d_oracle(pol, prec, case):
    p = CASES[case](pol)
    st, scale = _oracle_with_scales(p)
    with rk.Context2D(p, prec) as ctx:
        ctx.step(100)
        ctx.step(p.steps - 100)  # the DFT fold and the step index carry over between calls
        worst = {}
        for names in GROUPS[pol]:
            ref = {n: st.field(n, p) for n in names}
            peak = scale[names]
            for n in names:
                got = ctx.field(n)
                if peak == 0:
                    assert not np.any(got), n
                    continue
                worst[n] = np.abs(got - ref[n]).max() / peak
                assert worst[n] <= TOL[prec], (n, worst[n])
        X = ctx.spectra()
    worst["X"] = np.abs(X - st.X).max() / np.abs(st.X).max()
    assert worst["X"] <= TOL[prec], worst
    print(pol, prec, case, {k: f"{v:.1e}" for k, v in worst.items()})


@pytest.mark.parametrize("pol", ["tm", "te"])
def test_oblique_mode_rt_in_fp32_within_1e4_of_the_fp64_oracle(pol):
    p = _oblique(pol)
    st, _ = oracle.run2d(p)
    sv, _ = oracle.run2d(p.vacuum())
    Ro, To = oracle.reflection_transmission(st.X, sv.X)
    with rk.Context2D(p, "f32") as ctx:
        ctx.step(p.steps)
        X = ctx.spectra()
    with rk.Context2D(p.vacuum(), "f32") as ctx:
        ctx.step(p.steps)
        Xv = ctx.spectra()
    R, T = rk.rt(X, Xv)
    band = np.abs(sv.X[0]) >= 0.1 * np.abs(sv.X[0]).max()
    assert band.sum() > 50
    assert np.abs(R - Ro)[band].max() <= 1e-4 and np.abs(T - To)[band].max() <= 1e-4
