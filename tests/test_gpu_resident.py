"""The resident variant (one thread-block cluster holds a whole Mur-terminated slab for a whole DFT
block of steps) against the plain one-step-per-launch kernels, bit for bit: it performs the same
operations on the same values, so fields and spectra must be identical. Sizes cover both padding
cases (nz - 1 a multiple of the warp's cell span, where the left padding becomes 1), one and
several CTAs per cluster (small thread counts force the exchange between CTAs through distributed
shared memory at many cell positions), the source next to either end and in the middle, and
probes on the end cells."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _slab(nz, seed, src=None, steps=257):
    u = wl.uniform01(seed, 3 * nz)
    s = wl.c1_plain_slab(nz=max(nz, 16), steps=steps)
    s.nz = nz
    s.wp2 = (2 * np.pi * 60e9 * u[:nz]) ** 2 * (u[nz:2 * nz] > 0.3)
    s.nu = 1e11 * u[2 * nz:]
    s.src_cell = src if src is not None else 1 + (nz - 2) // 3
    s.probes = [0, nz - 1, nz // 2]
    s.src_tau = 4 * s.dt
    s.src_t0 = 3 * s.src_tau
    s.freq_hz = np.linspace(1e9, 1e12, 7)
    return s


def _run(s, prec, **opts):
    with rk.Context(s, prec, options=opts) as ctx:
        used = ctx.options()
        ctx.step(100)
        ctx.step(s.steps - 100)  # two calls: the second starts mid DFT block
        X = ctx.spectra()
        F = ctx.fields(0)
    return used, X, F


SIZES = {"f64": [8, 9, 13, 33, 63, 64, 65, 127, 129, 257, 511, 1000, 1537, 2047, 2048, 2049, 4097, 8191, 16383],
         "f32": [8, 9, 13, 33, 65, 127, 129, 257, 511, 1000, 2047, 2049, 4097, 16385, 32767]}


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resident_variant_is_bitwise_equal_to_the_plain_kernels(prec):
    for nz in SIZES[prec]:
        for src in (None, 1, nz - 2):
            s = _slab(nz, 7 * nz + (src or 0), src)
            base = _run(s, prec, variant=1)
            shapes = [{"variant": 0}, {"variant": 3}]
            small = 1 if prec == "f64" else 2
            if nz <= 32 * small * 16:  # up to 16 CTAs of one warp, fewest cells per thread
                shapes.append({"variant": 3, "res_threads": 32, "res_cells": small})
            if 64 < nz <= 64 * 2 * 16:
                shapes.append({"variant": 3, "res_threads": 64, "res_cells": 2})
            big = 8 if prec == "f64" else 16
            if 32 * big < nz <= 32 * big * 16:  # several CTAs of one warp, most cells per thread
                shapes.append({"variant": 3, "res_threads": 32, "res_cells": big})
            for opts in shapes:
                used, X, F = _run(s, prec, **opts)
                assert used["variant"] == 3, (nz, opts, used)
                assert np.array_equal(X, base[1]), (prec, nz, src, opts)
                for a, b in zip(F, base[2]):
                    assert np.array_equal(a, b), (prec, nz, src, opts)


def test_paper_slab_runs_resident_under_auto_and_matches_the_oracle():
    s = wl.c1_plain_slab()
    ref, ser = oracle.run1d(s, series=True)
    peak = np.abs(ser).max()
    for prec, tol in (("f64", 1e-12), ("f32", 1e-4)):
        used, X, F = _run(s, prec)
        assert used["variant"] == 3
        assert np.abs(X[0] - ref.X).max() <= tol * np.abs(ref.X).max()
        assert np.abs(F[0] - ref.E).max() <= (tol if prec == "f64" else 1e-3) * peak


def test_resident_variant_is_refused_where_it_does_not_apply():
    s = _slab(600, 3)
    cases = [([s, _slab(700, 4)], "f32", {}),  # a batch
             (_slab(16385, 5), "f64", {}),  # longer than 16 CTAs x 128 threads x 8 cells
             (_slab(32769, 6), "f32", {})]
    c = _slab(600, 7)
    c.bc, c.cpml_cells, c.probes = "cpml", 8, [8, 591]
    cases.append((c, "f64", {}))
    e2 = _slab(600, 8)
    e2.scheme = rk.RKETD_SCHEME_ETD2
    cases.append((e2, "f64", {}))
    for slabs, prec, extra in cases:
        with pytest.raises(rk.RketdError) as ei:
            rk.Context(slabs, prec, options={"variant": 3, **extra})
        assert ei.value.status == 6
        with rk.Context(slabs, prec) as ctx:  # auto falls back
            assert ctx.options()["variant"] in (1, 2)


def test_eq9_recursion_runs_resident_bitwise_equal_to_plain():
    s = _slab(1537, 11)
    s.scheme = rk.RKETD_SCHEME_ETD1
    for prec in ("f64", "f32"):
        base = _run(s, prec, variant=1)
        used, X, F = _run(s, prec)
        assert used["variant"] == 3
        assert np.array_equal(X, base[1])
        assert all(np.array_equal(a, b) for a, b in zip(F, base[2]))


def test_resident_graph_replay_timing_and_autotune_keep_results_bitwise():
    s = _slab(2000, 13, steps=1500)
    for prec in ("f64", "f32"):
        direct = _run(s, prec, use_graphs=2)
        with rk.Context(s, prec, options={"use_graphs": 1}) as ctx:
            for _ in range(2):
                ctx.reset()
                ctx.step(1500)
                assert np.array_equal(ctx.spectra(), direct[1])
            ctx.reset()
            ctx.kernel_timing(True)
            ctx.step(1500)
            ms, n, cells = ctx.get_kernel_timing()
            assert n > 0 and ms > 0 and cells == 2000 * 1500
            ctx.kernel_timing(False)
            assert np.array_equal(ctx.spectra(), direct[1])
        with rk.Context(s, prec) as ctx:
            ctx.step(700)
            ctx.autotune(2)
            ctx.step(800)
            assert np.array_equal(ctx.spectra(), direct[1])
            assert all(np.array_equal(a, b) for a, b in zip(ctx.fields(0), direct[2]))
