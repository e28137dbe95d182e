"""The 1D tile plan (rketd_plan_tiles_1d, host only): the temporally blocked step is correct only if
every cell is exact in exactly one tile, interior tiles load no boundary cell, and the tiles that
sample a probe or load a source cell run in the launch that has that code. Checked on seeded
random batches over the tile shapes, Mur and CPML ends, and slabs too short for an interior tile."""
import numpy as np
import pytest

from paper_1709_00821_gb300 import rketd as rk

SHAPES = [(8, 4), (8, 32), (12, 32), (16, 4), (16, 32), (16, 64), (32, 64)]


def _batch(rng, n_slabs, nc):
    nz = rng.integers(8 + 2 * nc, 6000, n_slabs)
    nz[: max(1, n_slabs // 4)] = rng.integers(8 + 2 * nc, 200 + 2 * nc, max(1, n_slabs // 4))  # short slabs
    src = np.array([rng.integers(nc + 1, n - nc - 1) for n in nz])
    n_probes = 3
    probes = np.array([rng.integers(0, n, n_probes) for n in nz])
    return nz, src, probes


def _edge_width(T):
    return 4 if 32 * 4 - 2 * T >= 32 else 8


@pytest.mark.parametrize("K,T", SHAPES)
@pytest.mark.parametrize("nc", [0, 16])
def test_tile_plan_covers_every_cell_once_and_keeps_interior_tiles_off_the_boundary(K, T, nc):
    rng = np.random.default_rng(1000 * K + 10 * T + nc)
    nz, src, probes = _batch(rng, 24, nc)
    rows = rk.plan_tiles_1d(nz, src, probes, nc, K, T)
    slab, start, vlo, vhi, kind, src_local, probe_count, loaded = rows.T
    # launch order: interior tiles without a probe or a source, then those with one, then edge tiles
    assert np.all(np.diff(kind) >= 0)
    L = 32 * K
    Le = 32 * _edge_width(T)
    assert np.all(loaded[kind < 2] == L) and np.all(loaded[kind == 2] == Le)
    for s in range(len(nz)):
        mine = slab == s
        hits = np.zeros(nz[s], dtype=np.int64)
        for st, lo, hi in zip(start[mine], vlo[mine], vhi[mine]):
            hits[st + lo:st + hi] += 1
        assert np.all(hits == 1), (s, np.flatnonzero(hits != 1)[:5])
        lo_guard, hi_guard = max(1, nc), nz[s] - 2 - nc
        inner = mine & (kind < 2)
        for st, lo, hi, k, sl, pcnt in zip(start[inner], vlo[inner], vhi[inner], kind[inner], src_local[inner],
                                           probe_count[inner]):
            assert st % 4 == 0  # 16-byte vector loads
            assert st >= lo_guard and st + L - 1 <= hi_guard  # no boundary cell loaded
            assert T <= lo < hi <= L - T  # exact cells after T steps
            loads_src = st <= src[s] < st + L
            assert sl == (src[s] - st if loads_src else -1)
            n_in = int(np.sum((probes[s] >= st + lo) & (probes[s] < st + hi)))
            assert pcnt == n_in
            assert (k == 1) == (loads_src or n_in > 0)
        # edge tiles take only the ends: the guard plus one tile's halo (and alignment) on the left, and
        # on the right the guard, the halo and a few cells after the shifted last interior tile
        if np.any(inner):
            ev = mine & (kind == 2)
            cells = np.zeros(nz[s], dtype=bool)
            for st, lo, hi in zip(start[ev], vlo[ev], vhi[ev]):
                cells[st + lo:st + hi] = True
            left = np.flatnonzero(cells[: nz[s] // 2])
            right = np.flatnonzero(cells[nz[s] // 2:])
            assert left.size <= lo_guard + T + 3
            assert right.size <= T + nc + 4


def test_tile_plan_rejects_bad_shapes_and_cells():
    nz, src, probes = np.array([2000]), np.array([100]), np.array([[300]])
    with pytest.raises(rk.RketdError):
        rk.plan_tiles_1d(nz, src, probes, 0, 6, 32)  # K not a multiple of 4
    with pytest.raises(rk.RketdError):
        rk.plan_tiles_1d(nz, src, probes, 0, 16, 30)  # T not a multiple of 4
    with pytest.raises(rk.RketdError):
        rk.plan_tiles_1d(nz, np.array([0]), probes, 0, 16, 32)  # source on the end cell
    with pytest.raises(rk.RketdError):
        rk.plan_tiles_1d(nz, src, np.array([[2000]]), 0, 16, 32)  # probe outside the slab
