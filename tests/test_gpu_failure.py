"""Failure paths, exercised without faulting the GPU.

* A staged-copy wait that gives up: the 3D staged form's compute threads are told to stop polling
  their mbarrier at once (a test hook), so every block gives up before its first copy lands, lets
  the copies it issued land (those waits keep their full bound), and reports through the context's
  status word; rketd_sync_3d returns RKETD_ETIMEOUT, and after a reset the same context reproduces
  a clean run bit for bit.
* An out-of-memory device: each device allocation the library makes while creating and running a
  1D, batched, 2D and 3D context is made to fail in turn (a host-side hook; the device is not
  touched). Every call that meets one returns RKETD_ENOMEM, nothing stays allocated, and the next
  context runs as before.
* Non-finite fields: a finite source amplitude that overflows FP32 (1e308) is reported by the
  finite scan as RKETD_ENUMERIC; a clean run passes it.
"""
import numpy as np
import pytest
import torch

from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl
from test_gpu_3d import _lean

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT, ENUMERIC = 3, 5, 7
E3 = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Jx", "Jy", "Jz")


def _lean_short(steps=40):
    p = _lean()
    p.steps = steps
    return p


def test_staged_wait_that_gives_up_reports_etimeout_and_the_context_recovers():
    p = _lean_short()
    with rk.Context3D(p, "f32", variant="staged") as ctx:
        ctx.step(p.steps)
        ctx.sync()
        ref = [ctx.field(n) for n in E3]
        Xref = ctx.spectra()
        ctx.reset()
        ctx.set_wait_limit(0)
        ctx.step(3)
        with pytest.raises(rk.RketdError) as ei:
            ctx.sync()
        assert ei.value.status == ETIMEOUT
        ctx.set_wait_limit(-1)
        ctx.reset()
        ctx.step(p.steps)
        ctx.sync()
        assert all(np.array_equal(ctx.field(n), r) for n, r in zip(E3, ref))
        assert np.array_equal(ctx.spectra(), Xref)


def _run_1d():
    s = wl.c1_plain_slab(nz=1 << 20, steps=600)
    with rk.Context(s, "f32") as ctx:
        ctx.step(s.steps)
        return [ctx.spectra(), *ctx.fields(0)]


def _run_batch():
    b = wl.c3_batch(subset=[0, 5, 17], steps=600)
    with rk.Context(b.slabs, "f32") as ctx:
        ctx.step(b.steps)
        return [ctx.spectra(), *ctx.fields(2)]


def _run_2d():
    p = wl.slab_2d(64, 400, "tm", mode=1, steps=300)
    with rk.Context2D(p, "f32") as ctx:
        ctx.step(p.steps)
        return [ctx.spectra(), ctx.field("Ez"), ctx.field("Jz")]


def _run_3d():
    p = _lean_short()
    with rk.Context3D(p, "f32", variant="staged") as ctx:
        ctx.step(p.steps)
        ctx.sync()
        return [ctx.spectra(), ctx.field("Ex"), ctx.field("Jx")]


RUNS = {"1d": _run_1d, "batch": _run_batch, "2d": _run_2d, "3d": _run_3d}


@pytest.mark.parametrize("kind", list(RUNS))
def test_each_device_allocation_failure_returns_enomem_and_leaks_nothing(kind):
    run = RUNS[kind]
    n0 = rk.debug_alloc_count()
    ref = run()
    n_alloc = rk.debug_alloc_count() - n0
    assert n_alloc > 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    enomem = 0
    for k in range(n_alloc):
        rk.debug_fail_alloc(k)
        try:
            got = run()
        except rk.RketdError as e:
            assert e.status == ENOMEM, (k, e)
            enomem += 1
        else:  # an allocation whose failure the library absorbs must leave the results unchanged
            assert all(np.array_equal(a, b) for a, b in zip(got, ref)), k
        finally:
            rk.debug_fail_alloc(-1)
    assert enomem >= n_alloc // 2, (enomem, n_alloc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)  # no context's memory stays behind
    got = run()
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))


def test_overflowing_source_is_reported_by_the_finite_scan():
    s = wl.c1_plain_slab(steps=300)
    with rk.Context(s, "f32") as ctx:
        ctx.step(s.steps)
        ctx.check_finite()  # a clean run passes
    s.src_amp = 1e308  # finite, validated, and beyond FP32
    with rk.Context(s, "f32") as ctx:
        ctx.step(s.steps)
        with pytest.raises(rk.RketdError) as ei:
            ctx.check_finite()
        assert ei.value.status == ENUMERIC
    p = wl.slab_2d(64, 200, "te", mode=1, steps=100)
    with rk.Context2D(p, "f32") as ctx:
        ctx.step(p.steps)
        ctx.check_finite()
    p.src_amp = 1e308
    with rk.Context2D(p, "f32") as ctx:
        ctx.step(p.steps)
        with pytest.raises(rk.RketdError) as ei:
            ctx.check_finite()
        assert ei.value.status == ENUMERIC
    q = _lean_short(30)
    with rk.Context3D(q, "f32", variant="staged") as ctx:
        ctx.step(q.steps)
        ctx.check_finite()
    q.src_amp = 1e308
    with rk.Context3D(q, "f32", variant="staged") as ctx:
        ctx.step(q.steps)
        with pytest.raises(rk.RketdError) as ei:
            ctx.check_finite()
        assert ei.value.status == ENUMERIC
