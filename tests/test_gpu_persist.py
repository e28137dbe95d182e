"""Persistent variant of the tiled step (options.variant = 4): every pass of a DFT block in one
launch, tiles waiting only for their slab's neighbouring tiles of the previous pass.

The arithmetic is the tiled variant's, so fields and spectra must agree with it bit for bit, for
ragged batches, for CPML and split-PML ends (edge tiles with memories), across DFT blocks, for a
step count that ends in a partial pass, and under CUDA-graph replay. The failure path (a wait
that gives up) is exercised with the wait limit set to zero: no GPU fault, a status word.
"""
import numpy as np
import pytest

from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _run(slabs, steps, **opts):
    with rk.Context(slabs, "f32", options=opts) as ctx:
        ctx.step(steps)
        ctx.sync()
        X = ctx.spectra()
        F = [ctx.fields(i) for i in range(len(slabs) if isinstance(slabs, list) else 1)]
    return X, F


def _same(a, b):
    Xa, Fa = a
    Xb, Fb = b
    assert np.array_equal(Xa, Xb)
    for fa, fb in zip(Fa, Fb):
        for u, v in zip(fa, fb):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("steps", [1024 + 96, 1300])
def test_ragged_batch_is_bitwise_the_tiled_variant(steps):
    """Eight slabs of the batch recipe (1 024 .. 65 536 cells), two probes and a source each, Mur
    ends; 1 300 steps end in a pass of 20 steps."""
    b = wl.c3_batch(subset=[0, 1, 2, 3, 17, 99, 1000, 4095], steps=steps)
    _same(_run(b.slabs, steps, variant=4), _run(b.slabs, steps, variant=2))


@pytest.mark.parametrize("K,T", [(16, 32), (8, 16), (12, 24)])
def test_tile_shapes_match_the_tiled_variant(K, T):
    b = wl.c3_batch(subset=[5, 6, 7], steps=700)
    opts = dict(cells_per_lane=K, tb_steps=T, dft_block=T * 16)
    _same(_run(b.slabs, 700, variant=4, **opts), _run(b.slabs, 700, variant=2, **opts))


@pytest.mark.parametrize("bc,n", [("cpml", 16), ("pml", 5)])
def test_absorbing_ends_with_memories_match_the_tiled_variant(bc, n):
    """Edge tiles with CPML memories (read and written every pass) or split-PML layers."""
    s = wl.c2_epstein(nz=20000, steps=600, nfreq=16)
    s.probes = [1200, 15000]
    s.src_cell = 600
    s.bc, s.cpml_cells = bc, n
    if bc == "pml":
        s.wp2 = np.where((np.arange(s.nz) < n) | (np.arange(s.nz) > s.nz - 1 - n), 0.0, s.wp2)
    _same(_run(s, 600, variant=4), _run(s, 600, variant=2))


def test_graph_replay_and_reset_reproduce_the_run():
    b = wl.c3_batch(subset=[10, 20, 30], steps=1024)
    with rk.Context(b.slabs, "f32", options={"variant": 4}) as ctx:
        out = []
        for _ in range(3):  # direct, captured, replayed
            ctx.reset()
            ctx.step(1024)
            ctx.sync()
            out.append((ctx.spectra(), [ctx.fields(i) for i in range(3)]))
    _same(out[0], out[1])
    _same(out[0], out[2])


def test_a_wait_that_gives_up_is_reported_and_the_context_recovers():
    b = wl.c3_batch(subset=[40, 41], steps=256)
    clean = _run(b.slabs, 256, variant=4)
    with rk.Context(b.slabs, "f32", options={"variant": 4}) as ctx:
        ctx.set_wait_limit(0)  # every wait gives up at once
        ctx.step(256)
        with pytest.raises(rk.RketdError) as e:
            ctx.sync()
        assert e.value.status == 5  # RKETD_ETIMEOUT
        ctx.set_wait_limit(-1)
        ctx.reset()
        ctx.step(256)
        ctx.sync()
        got = (ctx.spectra(), [ctx.fields(i) for i in range(2)])
    _same(got, clean)


def test_fp64_and_the_eq10_recursion_are_refused():
    s = wl.c1_plain_slab(steps=10)
    with pytest.raises(rk.RketdError) as e:
        rk.Context(s, "f64", options={"variant": 4})
    assert e.value.status == 6
    s.scheme = wl.SCHEME_ETD2
    with pytest.raises(rk.RketdError) as e:
        rk.Context(s, "f32", options={"variant": 4})
    assert e.value.status == 6


def test_autotune_keeps_the_persistent_variant():
    b = wl.c3_batch(subset=[1, 2, 3, 4], steps=512)
    with rk.Context(b.slabs, "f32", options={"variant": 4}) as ctx:
        ctx.autotune(passes=2)
        assert ctx.options()["variant"] == 4
        K, T = ctx.options()["cells_per_lane"], ctx.options()["tb_steps"]
    opts = dict(cells_per_lane=K, tb_steps=T)
    _same(_run(b.slabs, 512, variant=4, **opts), _run(b.slabs, 512, variant=2, **opts))
