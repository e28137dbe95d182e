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


@pytest.mark.parametrize("K,T", [(8, 16), (12, 32), (16, 32), (16, 8), (8, 28)])
def test_end_tile_plan_holds_each_mur_end_in_one_wide_tile(K, T):
    """end_tiles: slabs of at least 2 (32K - T) cells get no edge tiles; the tile that starts at 0
    holds [0, 32K - T) exactly, the one ending at round_up(nz, 4) - 1 holds its cells from T on,
    both run with the probe/source tiles; every cell is still exact in exactly one tile, and no
    other interior tile loads a boundary cell."""
    rng = np.random.default_rng(7 * K + T)
    L = 32 * K
    nz = np.concatenate([rng.integers(2 * (L - T), 12000, 20), [2 * (L - T) - 5, 2 * (L - T) + 1, L + 40, 100]])
    src = np.array([rng.integers(1, n - 1) for n in nz])
    probes = np.array([rng.integers(0, n, 3) for n in nz])
    rows = rk.plan_tiles_1d(nz, src, probes, 0, K, T, True)
    slab, start, vlo, vhi, kind, src_local, probe_count, loaded = rows.T
    assert np.all(np.diff(kind) >= 0)
    for s in range(len(nz)):
        mine = slab == s
        hits = np.zeros(nz[s], dtype=np.int64)
        for st, lo, hi in zip(start[mine], vlo[mine], vhi[mine]):
            hits[st + lo:st + hi] += 1
        assert np.all(hits == 1), (s, np.flatnonzero(hits != 1)[:5])
        ends = ((nz[s] + 3) // 4) * 4
        if ends - L + 2 * T - L >= 1:  # long enough for end tiles
            assert not np.any(mine & (kind == 2))
            left = mine & (start == 0)
            right = mine & (start + L - 1 >= nz[s] - 1)
            assert left.sum() == 1 and right.sum() == 1
            assert kind[left][0] == 1 and vlo[left][0] == 0 and vhi[left][0] == L - T
            assert kind[right][0] == 1 and start[right][0] == ends - L and vlo[right][0] == T
            assert vhi[right][0] == nz[s] - start[right][0]
            assert start[right][0] % 4 == 0 and start[right][0] + L <= ((nz[s] + 31) // 32) * 32  # inside storage
            inner = mine & ~left & ~right
            assert np.all(kind[inner] < 2) and np.all(loaded[mine] == L)
            assert np.all(start[inner] >= 1) and np.all(start[inner] + L - 1 <= nz[s] - 2)
            assert np.all(start[inner] % 4 == 0)
            assert np.all((vlo[inner] >= T) & (vhi[inner] <= L - T))
        else:  # short slabs keep the edge tiles
            assert np.any(mine & (kind == 2))
    # without end tiles every slab has edge tiles
    rows0 = rk.plan_tiles_1d(nz, src, probes, 0, K, T)
    assert all(np.any((rows0[:, 0] == s) & (rows0[:, 4] == 2)) for s in range(len(nz)))


def test_end_tiles_apply_to_mur_ends_only():
    """With CPML ends (cpml_cells > 0) the end-tile request changes nothing: the plan is the edge-tile
    plan, row for row."""
    rng = np.random.default_rng(99)
    nz = rng.integers(2000, 9000, 12)
    src = np.array([rng.integers(20, n - 20) for n in nz])
    probes = np.array([rng.integers(20, n - 20, 2) for n in nz])
    for K, T in ((16, 32), (12, 16)):
        assert np.array_equal(rk.plan_tiles_1d(nz, src, probes, 16, K, T, True),
                              rk.plan_tiles_1d(nz, src, probes, 16, K, T, False))

