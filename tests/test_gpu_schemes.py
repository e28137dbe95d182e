"""GPU parity of the two other current recursions of Sec. II against the FP64 oracle: the
first-order ETD of Eq. 9 (a change of the update coefficients only, run by every kernel) and
Eq. 10 read literally (explicit second-order ETD, which carries E^{n-1} and runs on the plain
kernels). Tolerances as for the Eq. 11 path: FP64 spectra within 1e-12 of their peak, fields
within 1e-12 of the run's field scale; FP32 spectra within 1e-4 of their peak over the whole band
and R/T within 1e-4 absolute where the incident spectrum holds at least 6% of its peak."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _with(slab, scheme):
    slab.scheme = scheme
    return slab


def _run(slab, prec, steps=None, **opts):
    first = slab[0] if isinstance(slab, list) else slab
    with rk.Context(slab, prec, options=opts or None) as ctx:
        ctx.step(first.steps if steps is None else steps)
        X = ctx.spectra()
        fields = [ctx.fields(i) for i in range(ctx.n_slabs)]
        used = ctx.options()
    return X, fields, used


@pytest.fixture(scope="module", params=[1, 2], ids=["eq9", "eq10"])
def paper_slab(request):
    s = _with(wl.c1_plain_slab(), request.param)
    tot, ser = oracle.run1d(s, series=True)
    inc, _ = oracle.run1d(s.vacuum())
    return s, tot, inc, np.abs(ser).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paper_slab_matches_the_oracle(paper_slab, prec):
    s, tot, inc, peak = paper_slab
    variants = [1, 2] if s.scheme == 1 else [0, 1]  # Eq. 10: auto selects plain
    for v in variants:
        X, fields, used = _run(s, prec, variant=v)
        Xv, _, _ = _run(s.vacuum(), prec, variant=v)
        if s.scheme == 2:
            assert used["variant"] == 1
        E, H, J = fields[0]
        eX = np.abs(X[0] - tot.X).max() / np.abs(tot.X).max()
        eXv = np.abs(Xv[0] - inc.X).max() / np.abs(inc.X).max()
        R, T = rk.rt(X[0], Xv[0])
        Ro, To = oracle.reflection_transmission(tot.X, inc.X)
        if prec == "f64":
            eta0 = np.sqrt(wl.MU0 / wl.EPS0)
            assert eX <= 1e-12 and eXv <= 1e-12, (v, eX, eXv)
            assert np.abs(E - tot.E).max() <= 1e-12 * peak
            assert np.abs(H - tot.H).max() * eta0 <= 1e-12 * peak
            assert np.abs(J - tot.J).max() * s.dt / wl.EPS0 <= 1e-12 * peak
            band = s.freq_hz >= 2.5e9
            assert np.abs(R - Ro)[band].max() <= 1e-12 * np.abs(Ro).max()
            assert np.abs(T - To)[band].max() <= 1e-12 * np.abs(To).max()
        else:
            assert eX <= 1e-4 and eXv <= 1e-4, (v, eX, eXv)
            band = s.freq_hz >= 3e9
            assert np.abs(R - Ro)[band].max() <= 1e-4 and np.abs(T - To)[band].max() <= 1e-4
        print(s.scheme, prec, v, f"spectra {eX:.2e}")


def _random_slab(nz, seed, scheme, bc="mur", cpml=0, steps=211):
    u = wl.uniform01(seed, 3 * nz)
    s = wl.c1_plain_slab(nz=max(nz, 16), steps=steps)
    s.nz = nz
    s.wp2 = (2 * np.pi * 60e9 * u[:nz]) ** 2 * (u[nz:2 * nz] > 0.3)
    s.nu = 1e11 * u[2 * nz:]
    s.bc, s.cpml_cells = bc, cpml
    lo = max(1, cpml)
    s.src_cell = lo + (nz - 2 * lo) // 3
    s.probes = [lo, nz - 1 - lo] if bc == "cpml" else [0, nz - 1]
    s.src_tau = 4 * s.dt
    s.src_t0 = 3 * s.src_tau
    s.freq_hz = np.linspace(1e9, 1e12, 7)
    s.scheme = scheme
    return s


@pytest.mark.parametrize("bc", ["mur", "cpml"])
@pytest.mark.parametrize("scheme", [1, 2])
def test_random_media_match_the_oracle_and_eq9_tiles_equal_plain_bitwise(scheme, bc):
    """Random plasma in every cell, CPML or Mur ends, several grid sizes (ragged tails). Eq. 9: the
    tiled kernels (FP64 and FP32 pairs and scalar) give the plain kernels' fields bit for bit."""
    for nz in (40, 97, 545, 3001):
        s = _random_slab(nz, 3 * nz + scheme, scheme, bc, 6 if bc == "cpml" else 0)
        ref, _ = oracle.run1d(s)
        X, fields, _ = _run(s, "f64", variant=1)
        E, H, J = fields[0]
        rel = lambda a, b: np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert rel(E, ref.E) <= 1e-12 and rel(H, ref.H) <= 1e-12 and rel(J, ref.J) <= 1e-12, nz
        assert rel(X[0], ref.X) <= 1e-12, nz
        if scheme == 1:
            for prec, tiles in (("f64", [(4, 8), (8, 4)]), ("f32", [(8, 12), (16, 32)])):
                base = _run(s, prec, variant=1)
                for K, T in tiles:
                    for pairs in ((0, 2) if prec == "f32" else (0,)):
                        got = _run(s, prec, variant=2, cells_per_lane=K, tb_steps=T, fp32_pairs=pairs)
                        assert np.array_equal(got[0], base[0]), (prec, K, T, pairs)
                        for a, b in zip(got[1][0], base[1][0]):
                            assert np.array_equal(a, b), (prec, K, T, pairs)


@pytest.mark.parametrize("scheme", [1, 2])
def test_ragged_batch_matches_per_slab_oracle(scheme):
    b = wl.c3_batch(subset=[0, 5, 17, 99, 1000], steps=2500)
    slabs = [_with(s, scheme) for s in b.slabs]
    refs = [oracle.run1d(s)[0] for s in slabs]
    for prec, tol in (("f64", 1e-12), ("f32", 5e-4)):
        X, fields, _ = _run(slabs, prec)
        for i, ref in enumerate(refs):
            assert np.abs(X[i] - ref.X).max() <= tol * np.abs(ref.X).max(), (prec, i)
            assert np.abs(fields[i][0] - ref.E).max() <= tol * np.abs(ref.E).max(), (prec, i)


def test_eq10_state_file_carries_the_previous_field_and_resumes_bitwise():
    s = _with(wl.c1_plain_slab(steps=1500), 2)
    full = _run(s, "f64")
    with rk.Context(s, "f64") as ctx:
        ctx.step(700)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "st.bin")
            ctx.save(path)
            ctx.step(300)  # move on, then go back
            ctx.load(path)
        ctx.step(800)
        X = ctx.spectra()
        E, H, J = ctx.fields(0)
    assert np.array_equal(X, full[0])
    for a, b in zip((E, H, J), full[1][0]):
        assert np.array_equal(a, b)


def test_unsupported_combinations_are_refused():
    s = _with(wl.c1_plain_slab(steps=10), 2)
    with pytest.raises(rk.RketdError) as ei:
        rk.Context(s, "f32", options={"variant": 2})
    assert ei.value.status == 6
    with rk.Context(s, "f32") as ctx:
        with pytest.raises(rk.RketdError) as ei:
            ctx.autotune(1)
        assert ei.value.status == 6
    s1 = _with(wl.c1_plain_slab(steps=10), 1)
    with rk.Context(s1, "f32") as ctx:
        with pytest.raises(rk.RketdError) as ei:
            ctx.forward_ckpt(64, 16)
        assert ei.value.status == 6
