"""GPU parity of the paper's split-field PML ends (5 cells at both ends, Sec. III and Sec. IV.B)
against the FP64 oracle, on the paper's slab and on random media with ragged grid sizes; the tiled
and plain kernels agree bit for bit. Tolerances as for the other ends: FP64 spectra and fields
within 1e-12 of their peaks, R/T within 1e-12 of their peak from 2.5 GHz; FP32 spectra within 1e-4
of their peak and R/T within 1e-4 absolute from 3 GHz."""
import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pml(s, n=5):
    s.bc, s.cpml_cells = "pml", n
    return s


def _run(slabs, prec, steps, **opts):
    with rk.Context(slabs, prec, options=opts or None) as ctx:
        ctx.step(steps)
        X = ctx.spectra()
        F = [ctx.fields(i) for i in range(ctx.n_slabs)]
        used = ctx.options()
    return X, F, used


@pytest.fixture(scope="module")
def paper_slab():
    s = _pml(wl.c1_plain_slab())
    tot, ser = oracle.run1d(s, series=True)
    inc, _ = oracle.run1d(s.vacuum())
    return s, tot, inc, np.abs(ser).max()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paper_slab_with_split_pml_ends_matches_the_oracle(paper_slab, prec, variant):
    s, tot, inc, peak = paper_slab
    X, F, used = _run(s, prec, s.steps, variant=variant)
    Xv, _, _ = _run(s.vacuum(), prec, s.steps, variant=variant)
    assert used["variant"] in (1, 2)  # the resident variant takes Mur ends only
    E, H, J = F[0]
    eX = np.abs(X[0] - tot.X).max() / np.abs(tot.X).max()
    eXv = np.abs(Xv[0] - inc.X).max() / np.abs(inc.X).max()
    R, T = rk.rt(X[0], Xv[0])
    Ro, To = oracle.reflection_transmission(tot.X, inc.X)
    if prec == "f64":
        eta0 = np.sqrt(wl.MU0 / wl.EPS0)
        assert eX <= 1e-12 and eXv <= 1e-12, (eX, eXv)
        assert np.abs(E - tot.E).max() <= 1e-12 * peak
        assert np.abs(H - tot.H).max() * eta0 <= 1e-12 * peak
        band = s.freq_hz >= 2.5e9
        assert np.abs(R - Ro)[band].max() <= 1e-12 * np.abs(Ro).max()
        assert np.abs(T - To)[band].max() <= 1e-12 * np.abs(To).max()
    else:
        assert eX <= 1e-4 and eXv <= 1e-4, (eX, eXv)
        band = s.freq_hz >= 3e9
        assert np.abs(R - Ro)[band].max() <= 1e-4 and np.abs(T - To)[band].max() <= 1e-4


def _random_slab(nz, seed, n, steps=233):
    u = wl.uniform01(seed, 3 * nz)
    s = wl.c1_plain_slab(nz=max(nz, 16), steps=steps)
    s.nz = nz
    s.wp2 = (2 * np.pi * 60e9 * u[:nz]) ** 2 * (u[nz:2 * nz] > 0.3)
    s.nu = 1e11 * u[2 * nz:]
    s.wp2[:n] = 0.0
    s.wp2[nz - n:] = 0.0
    s.src_cell = n + (nz - 2 * n) // 3
    s.probes = [n, nz - 1 - n]
    s.src_tau = 4 * s.dt
    s.src_t0 = 3 * s.src_tau
    s.freq_hz = np.linspace(1e9, 1e12, 7)
    return _pml(s, n)


def test_random_media_with_split_pml_ends_match_the_oracle_and_tiles_equal_plain_bitwise():
    for nz, n in ((16, 5), (40, 5), (97, 3), (545, 5), (3001, 8), (4097, 1)):
        s = _random_slab(nz, 11 * nz + n, n)
        ref, _ = oracle.run1d(s)
        X, F, _ = _run(s, "f64", s.steps, variant=1)
        E, H, J = F[0]
        rel = lambda a, b: np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert rel(E, ref.E) <= 1e-12 and rel(H, ref.H) <= 1e-12 and rel(J, ref.J) <= 1e-12, nz
        assert rel(X[0], ref.X) <= 1e-12, nz
        for prec, shapes in (("f64", [(4, 8), (8, 4)]), ("f32", [(8, 12), (16, 32)])):
            base = _run(s, prec, s.steps, variant=1)
            for K, T in shapes:
                for pairs in ((0, 2) if prec == "f32" else (0,)):
                    got = _run(s, prec, s.steps, variant=2, cells_per_lane=K, tb_steps=T, fp32_pairs=pairs)
                    assert np.array_equal(got[0], base[0]), (nz, prec, K, T)
                    assert all(np.array_equal(a, b) for a, b in zip(got[1][0], base[1][0])), (nz, prec, K, T)


def test_ragged_batch_with_split_pml_ends_matches_per_slab_oracle():
    b = wl.c3_batch(subset=[1, 7, 300, 2048], steps=2500)
    slabs = [_pml(s) for s in b.slabs]
    refs = [oracle.run1d(s)[0] for s in slabs]
    for prec, tol in (("f64", 1e-12), ("f32", 5e-4)):
        X, F, _ = _run(slabs, prec, b.steps)
        for i, ref in enumerate(refs):
            assert np.abs(X[i] - ref.X).max() <= tol * np.abs(ref.X).max(), (prec, i)
            assert np.abs(F[i][0] - ref.E).max() <= tol * np.abs(ref.E).max(), (prec, i)


def test_resident_variant_refuses_pml_ends():
    s = _pml(wl.c1_plain_slab(steps=10))
    with pytest.raises(rk.RketdError) as ei:
        rk.Context(s, "f64", options={"variant": 3})
    assert ei.value.status == 6
