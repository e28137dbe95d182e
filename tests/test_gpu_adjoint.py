"""GPU adjoint (through the C ABI) against the FP64 oracle adjoint, which the CPU tests pin
to central finite differences. FP64: 1e-9 of the largest gradient; FP32: 1e-3 relative in norm."""
import numpy as np
import pytest

import oracle
from paper_1709_00821_gb300 import rketd as rk
from paper_1709_00821_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem(i=0, nz=700, steps=1600, region=(300, 400)):
    s = wl.c1_plain_slab(nz=nz, steps=steps)
    s.src_cell, s.probes = 100, [150, 600]
    s.freq_hz = np.linspace(5e9, 100e9, 24)
    base = wl.c4_profile(i, nz=nz, region=region, steps=steps)
    s.wp2, s.nu = base.wp2.copy(), base.nu.copy()
    tgt = wl.c4_profile(i + 1000, nz=nz, region=region, steps=steps)
    return s, tgt


def _oracle_case(s, tgt):
    inc, _ = oracle.run1d(s.vacuum())
    t = s.vacuum()
    t.wp2, t.nu = tgt.wp2.copy(), tgt.nu.copy()
    tt, _ = oracle.run1d(t)
    R_t = np.abs((tt.X[0] - inc.X[0]) / inc.X[0])
    tot, _ = oracle.run1d(s)
    L, gX = oracle.reflection_loss(tot.X, inc.X, R_t)
    gw, gn = oracle.adjoint(s, gX)
    return inc, R_t, gX, gw, gn


def _gpu_grad(slabs, prec, gX, window, every, steps, **opts):
    import torch

    with rk.Context(slabs, prec, options=opts or None) as ctx:
        ctx.forward_ckpt(steps, every)
        X = ctx.spectra()
        n = sum(s.nz for s in slabs)
        gw = torch.zeros(n, dtype=torch.float64, device="cuda")
        gn = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.adjoint(np.ascontiguousarray(gX.real), np.ascontiguousarray(gX.imag), window[0], window[1], gw, gn)
        ctx.sync()
        return X, gw.cpu().numpy(), gn.cpu().numpy()


@pytest.fixture(scope="module")
def case():
    s, tgt = _problem()
    return s, _oracle_case(s, tgt)


@pytest.mark.parametrize("every", [256, 512, 1600, 333])
def test_fp64_adjoint_matches_oracle_adjoint(case, every):
    s, (inc, R_t, gX, gw_o, gn_o) = case
    X, gw, gn = _gpu_grad([s], "f64", gX[None], (300, 400), every, s.steps)
    w = slice(300, 400)
    assert np.abs(gw[w] - gw_o[w]).max() <= 1e-9 * np.abs(gw_o).max()
    assert np.abs(gn[w] - gn_o[w]).max() <= 1e-9 * np.abs(gn_o).max()
    assert not np.any(gw[:300]) and not np.any(gw[400:])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-3)])
def test_adjoint_with_the_source_cell_inside_the_trainable_window(prec, tol):
    """The plasma covers the source cell (da != 0 there) and the window contains it: the source
    also folds into the carried current, which gives the source cell's gradient a term of its own."""
    s, tgt = _problem(region=(60, 400))
    assert s.wp2[s.src_cell] > 0
    inc, R_t, gX, gw_o, gn_o = _oracle_case(s, tgt)
    X, gw, gn = _gpu_grad([s], prec, gX[None], (80, 400), 512, s.steps)
    w = slice(80, 400)
    if prec == "f64":
        assert np.abs(gw[w] - gw_o[w]).max() <= tol * np.abs(gw_o).max()
        assert np.abs(gn[w] - gn_o[w]).max() <= tol * np.abs(gn_o).max()
        k = s.src_cell
        assert abs(gw[k] - gw_o[k]) <= 1e-9 * abs(gw_o[k]) + 1e-12 * np.abs(gw_o).max()
    else:
        assert np.linalg.norm(gw[w] - gw_o[w]) <= tol * np.linalg.norm(gw_o[w])
        assert np.linalg.norm(gn[w] - gn_o[w]) <= tol * np.linalg.norm(gn_o[w])
    assert not np.any(gw[:80]) and not np.any(gw[400:])


def test_fp32_adjoint_within_1e3_of_oracle(case):
    s, (inc, R_t, gX, gw_o, gn_o) = case
    X, gw, gn = _gpu_grad([s], "f32", gX[None], (300, 400), 512, s.steps)
    w = slice(300, 400)
    assert np.linalg.norm(gw[w] - gw_o[w]) <= 1e-3 * np.linalg.norm(gw_o[w])
    assert np.linalg.norm(gn[w] - gn_o[w]) <= 1e-3 * np.linalg.norm(gn_o[w])


def test_batched_adjoint_gives_each_profile_its_own_gradient():
    slabs, refs = [], []
    for i in range(3):
        s, tgt = _problem(i)
        slabs.append(s)
        refs.append(_oracle_case(s, tgt))
    gX = np.stack([r[2] for r in refs])
    X, gw, gn = _gpu_grad(slabs, "f64", gX, (300, 400), 400, slabs[0].steps)
    for i, r in enumerate(refs):
        o = i * slabs[0].nz
        w = slice(o + 300, o + 400)
        assert np.abs(gw[w] - r[3][300:400]).max() <= 1e-9 * np.abs(r[3]).max()
        assert np.abs(gn[w] - r[4][300:400]).max() <= 1e-9 * np.abs(r[4]).max()


def test_autograd_function_drives_the_adjoint():
    import torch

    from paper_1709_00821_gb300.autograd import SpectraEngine

    s, tgt = _problem()
    inc, R_t, gX, gw_o, gn_o = _oracle_case(s, tgt)
    eng = SpectraEngine([s], "f64", steps=s.steps, ckpt_every=512, window=(300, 400))
    wp2 = torch.tensor(s.wp2, device="cuda", requires_grad=True)
    nu = torch.tensor(s.nu, device="cuda", requires_grad=True)
    xr, xi = eng(wp2, nu)
    inc_t = torch.tensor(inc.X[0], device="cuda")
    d = torch.complex(xr[0, 0], xi[0, 0]) - inc_t
    absr = torch.abs(d) / torch.abs(inc_t)
    loss = ((absr - torch.tensor(R_t, device="cuda")) ** 2).sum()
    loss.backward()
    eng.close()
    w = slice(300, 400)
    assert np.abs(wp2.grad.cpu().numpy()[w] - gw_o[w]).max() <= 1e-9 * np.abs(gw_o).max()
    assert np.abs(nu.grad.cpu().numpy()[w] - gn_o[w]).max() <= 1e-9 * np.abs(gn_o).max()


def test_unaligned_window_reaching_the_last_interior_cell():
    """Window [301, 699): not 4-aligned, ends at nz - 1 (record rows pad past the slab end)."""
    s, tgt = _problem(2, region=(301, 699))
    inc, R_t, gX, gw_o, gn_o = _oracle_case(s, tgt)
    X, gw, gn = _gpu_grad([s], "f64", gX[None], (301, 699), 512, s.steps)
    w = slice(301, 699)
    assert np.abs(gw[w] - gw_o[w]).max() <= 1e-9 * np.abs(gw_o).max()
    assert np.abs(gn[w] - gn_o[w]).max() <= 1e-9 * np.abs(gn_o).max()


def test_fp32_paired_adjoint_is_bitwise_equal_to_scalar(case):
    s, (inc, R_t, gX, gw_o, gn_o) = case
    a = _gpu_grad([s], "f32", gX[None], (300, 400), 512, s.steps)
    b = _gpu_grad([s], "f32", gX[None], (300, 400), 512, s.steps, fp32_pairs=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
