"""rketd_advance_1d_noalloc: the step entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: frameworks whose caching allocator owns the whole GPU,
loops that cannot pay for the device-wide synchronisation of an allocation. The entry point keeps its working memory
in a fixed array inside the library and only touches the caller's arrays. These tests
check it against the context API (rketd_create_1d + rketd_step + rketd_get_fields) on
two calls in a row, with the tolerances the other parity tests use.

This file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl


def _scales(slab):
    eta0 = math.sqrt(wl.MU0 / wl.EPS0)
    return 1.0, eta0, slab.dt / wl.EPS0  # E, H and J into the same normalised units


def _plasma_source(src):
    """c1 line with plasma everywhere, so that the source cell folds into the carried current."""
    slab = wl.c1_plain_slab()
    slab.wp2 = np.full(slab.nz, (2 * math.pi * 30e9) ** 2)
    slab.nu = np.full(slab.nz, 2e10)
    slab.src_cell = src
    return slab


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol,src", [("f64", 1e-12, None), ("f32", 1e-5, None),
                                          ("f64", 1e-12, 255), ("f64", 1e-12, 8), ("f32", 1e-5, 460),
                                          ("f32", 1e-5, 484), ("f32", 1e-5, 36)])
def test_noalloc_advance_matches_context_api_on_two_calls_in_a_row(prec, tol, src):
    """src None: the c1 slab (source in vacuum); otherwise a plasma line with the source cell where
    two interior tiles load it (or at the first interior cell)."""
    import torch

    slab = wl.c1_plain_slab() if src is None else _plasma_source(src)
    n1, n2 = 1500, 1337
    with rk.Context(slab, prec) as ctx:
        ctx.step(n1)
        ref1 = ctx.fields(0)
        ctx.step(n2)
        ref2 = ctx.fields(0)

    fdt = torch.float64 if prec == "f64" else torch.float32
    wp2 = torch.tensor(slab.wp2, dtype=torch.float64, device="cuda")
    nu = torch.tensor(slab.nu, dtype=torch.float64, device="cuda")
    E = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    H = torch.zeros(slab.nz - 1, dtype=fdt, device="cuda")
    J = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    ptrs = (E.data_ptr(), H.data_ptr(), J.data_ptr())

    rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), 0, n1, *ptrs)
    torch.cuda.synchronize()
    got1 = [t.double().cpu().numpy() for t in (E, H, J)]
    rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), n1, n2, *ptrs)
    torch.cuda.synchronize()
    got2 = [t.double().cpu().numpy() for t in (E, H, J)]

    for got, ref in ((got1, ref1), (got2, ref2)):
        scale = np.abs(ref[0]).max()
        assert scale > 1e-3
        for g, r, k in zip(got, ref, _scales(slab)):
            assert np.abs(g - r).max() * k <= tol * scale


@pytest.mark.gpu
@pytest.mark.parametrize("prec,nz", [("f32", 516), ("f32", 517), ("f32", 964), ("f32", 965), ("f32", 131072),
                                     ("f64", 260), ("f64", 261), ("f64", 508), ("f64", 509), ("f64", 131072)])
def test_noalloc_tiling_at_the_capacity_and_where_the_interior_tile_count_changes(prec, nz):
    """nz values on both sides of each change of the interior tile count (FP32: K = 16, 32 steps per
    pass, one more tile every 448 cells from 517; FP64: K = 8, 4 steps, every 248 from 261), and the
    largest slab the fixed array holds."""
    import torch

    slab = wl.c1_plain_slab(nz=nz, steps=1)
    slab.wp2 = np.full(nz, (2 * math.pi * 30e9) ** 2)
    slab.nu = np.full(nz, 2e10)
    slab.src_cell = nz // 3
    slab.probes = []
    n1 = 300
    with rk.Context(slab, prec) as ctx:
        ctx.step(n1)
        ref = ctx.fields(0)
    fdt = torch.float64 if prec == "f64" else torch.float32
    wp2 = torch.tensor(slab.wp2, dtype=torch.float64, device="cuda")
    nu = torch.tensor(slab.nu, dtype=torch.float64, device="cuda")
    E = torch.zeros(nz, dtype=fdt, device="cuda")
    H = torch.zeros(nz - 1, dtype=fdt, device="cuda")
    J = torch.zeros(nz, dtype=fdt, device="cuda")
    rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), 0, n1, E.data_ptr(), H.data_ptr(), J.data_ptr())
    torch.cuda.synchronize()
    got = [t.double().cpu().numpy() for t in (E, H, J)]
    tol = 1e-12 if prec == "f64" else 1e-5
    scale = np.abs(ref[0]).max()
    assert scale > 1e-3
    for g, r, k in zip(got, ref, _scales(slab)):
        assert np.abs(g - r).max() * k <= tol * scale


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_runs_the_first_order_recursion_like_the_context_api(prec, tol):
    """The Eq. 9 recursion is a change of coefficients only, which this entry point also takes."""
    import torch

    slab = _plasma_source(460)
    slab.scheme = rk.RKETD_SCHEME_ETD1
    n1 = 900
    with rk.Context(slab, prec) as ctx:
        ctx.step(n1)
        ref = ctx.fields(0)
    fdt = torch.float64 if prec == "f64" else torch.float32
    wp2 = torch.tensor(slab.wp2, dtype=torch.float64, device="cuda")
    nu = torch.tensor(slab.nu, dtype=torch.float64, device="cuda")
    E = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    H = torch.zeros(slab.nz - 1, dtype=fdt, device="cuda")
    J = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), 0, n1, E.data_ptr(), H.data_ptr(), J.data_ptr())
    torch.cuda.synchronize()
    got = [t.double().cpu().numpy() for t in (E, H, J)]
    scale = np.abs(ref[0]).max()
    assert scale > 1e-3
    for g, r, k in zip(got, ref, _scales(slab)):
        assert np.abs(g - r).max() * k <= tol * scale


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_call_recorded_into_a_cuda_graph_replays_like_the_context_api(prec, tol):
    """The call recorded into a CUDA graph (after one eager call, which looks up the fixed array's
    address) and replayed twice from the same starting state gives the context API's fields both
    times: it allocates nothing, synchronises nothing and reads its arguments at replay."""
    import torch

    slab = _plasma_source(255)
    n = 1024
    with rk.Context(slab, prec) as ctx:
        ctx.step(n)
        ref = ctx.fields(0)

    fdt = torch.float64 if prec == "f64" else torch.float32
    wp2 = torch.tensor(slab.wp2, dtype=torch.float64, device="cuda")
    nu = torch.tensor(slab.nu, dtype=torch.float64, device="cuda")
    E = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    H = torch.zeros(slab.nz - 1, dtype=fdt, device="cuda")
    J = torch.zeros(slab.nz, dtype=fdt, device="cuda")
    ptrs = (E.data_ptr(), H.data_ptr(), J.data_ptr())
    rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), 0, 1, *ptrs)  # eager warm-up call
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rk.advance_1d_noalloc(slab, prec, wp2.data_ptr(), nu.data_ptr(), 0, n, *ptrs)
    scale = np.abs(ref[0]).max()
    assert scale > 1e-3
    for _ in range(2):
        for t in (E, H, J):
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        got = [t.double().cpu().numpy() for t in (E, H, J)]
        for g, r, k in zip(got, ref, _scales(slab)):
            assert np.abs(g - r).max() * k <= tol * scale


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_tile_list_covers_every_cell_once_and_matches_its_launches(prec):
    """The tile list the entry point writes on the device, computed on the host by the same code:
    for slab lengths from 8 cells to the capacity (and where the interior tile count changes) and
    sources anywhere, every cell is exact in exactly one tile; the first launch's interior tiles
    load neither a boundary cell nor the source cell, the second launch's load the source cell,
    the third launch holds the edge tiles. Runs without a GPU."""
    rng = np.random.default_rng(17 if prec == "f32" else 18)
    K, T = (16, 32) if prec == "f32" else (8, 4)
    L, W = 32 * K, 32 * K - 2 * T
    a = ((1 + T + 3) // 4) * 4
    lengths = [8, 9, 31, 100, L + 3, a - T + L + 1, a - T + L + 2, a - T + L + W + 1, a - T + L + W + 2, 131072]
    lengths += list(rng.integers(8, 131073, 40))
    for nz in lengths:
        nz = int(nz)
        for src in {1, 2, nz // 2, nz - 3, nz - 2, int(rng.integers(1, nz - 1))}:
            rows, counts = rk.noalloc_tiles_1d(prec, nz, src)
            start, vlo, vhi, src_local, loaded = rows.T
            assert len(rows) == counts.sum() <= 4096
            hits = np.zeros(nz, dtype=np.int64)
            for st, lo, hi in zip(start, vlo, vhi):
                hits[st + lo:st + hi] += 1
            assert np.all(hits == 1), (nz, src, np.flatnonzero(hits != 1)[:5])
            n_main, n_src, n_edge = counts
            inner = slice(0, n_main + n_src)
            assert np.all(loaded[inner] == L) and np.all(loaded[n_main + n_src:] == 32 * 4)
            assert np.all(start[inner] >= 1) and np.all(start[inner] + L - 1 <= nz - 2)
            assert np.all(start[inner] % 4 == 0)
            loads_src = (start <= src) & (src < start + loaded)
            assert not np.any(loads_src[:n_main]) and np.all(loads_src[n_main:n_main + n_src])
            assert np.all(src_local == np.where(loads_src, src - start, -1))


def test_noalloc_rejects_slabs_beyond_the_fixed_capacity():
    """Checked before any device work: runs without a GPU."""
    slab = wl.c1_plain_slab(nz=131073, steps=1)
    slab.src_cell, slab.probes = 100, []
    with pytest.raises(rk.RketdError) as ei:
        rk.advance_1d_noalloc(slab, "f64", 1, 1, 0, 1, 1, 1, 1, stream=0)
    assert ei.value.status == 1
    assert "131072" in str(ei.value)
