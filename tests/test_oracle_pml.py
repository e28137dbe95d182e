"""Pins of the oracle's split-field PML (the paper's boundary, Sec. III and Sec. IV.B: 5 cells at both
ends), CPU only. In 1D only the z-split field exists, so the layer is one graded lossy layer with
matched electric and magnetic conductivities advanced by exponential differencing, backed by PEC walls;
the grading (m = 3, sigma_max = 0.8 (m + 1)/(eta0 dz)) is our reading, the paper gives none.

* the running-DFT R/T of the paper's slab with 5-cell PML ends converge to the exact steady-state
  response of the lattice including the layers (analytic.domain_response_pml, its own statement of
  the layer's update);
* the layer's reflection, against a domain whose ends are out of reach, stays below 2e-3 of the
  incident peak (8.9e-4 measured; first-order Mur reflects 2.1e-3 there);
* a planted mistake (no magnetic conductivity: an unmatched layer) fails the lattice pin;
* the layer must be vacuum (the oracle refuses plasma in it).
"""
import numpy as np
import pytest

import analytic as an
import oracle
from paper_1709_00821_gb300 import workloads as wl


def _pml_slab(steps, n=5, nz=2000):
    s = wl.c1_plain_slab(nz=nz, steps=steps)
    s.bc, s.cpml_cells = "pml", n
    return s


def _rt(s, **kw):
    st, _ = oracle.run1d(s, **kw)
    sv, _ = oracle.run1d(s.vacuum(), **kw)
    return oracle.reflection_transmission(st.X, sv.X)


@pytest.fixture(scope="module")
def lattice_rt():
    s = _pml_slab(1)
    m, smax, _, _ = oracle.cpml_defaults(s.dz)
    args = (s.dz, s.dt, s.freq_hz, s.src_cell, s.probes, s.cpml_cells, m, smax)
    tot = an.domain_response_pml(s.wp2, s.nu, *args)
    inc = an.domain_response_pml(np.zeros(s.nz), np.zeros(s.nz), *args)
    return (tot[:, 0] - inc[:, 0]) / inc[:, 0], tot[:, 1] / inc[:, 1]


def test_rt_with_split_pml_ends_converge_to_the_lattice_response(lattice_rt):
    Rd, Td = lattice_rt
    R8, T8 = _rt(_pml_slab(8000))
    R16, T16 = _rt(_pml_slab(16000))
    e8 = max(np.abs(R8 - Rd).max(), np.abs(T8 - Td).max())
    e16 = max(np.abs(R16 - Rd).max(), np.abs(T16 - Td).max())
    assert e16 < 1e-4 and e16 < e8 / 50, (e8, e16)
    hi = slice(70, None)
    assert max(np.abs(R16 - Rd)[hi].max(), np.abs(T16 - Td)[hi].max()) < 1e-7
    # the layers' reflection shows against the infinite lattice (no boundary at all)
    Ri, Ti = an.slab_rt_lattice(*(lambda s: (s.wp2, s.nu, s.dz, s.dt, s.freq_hz, s.probes[0], s.probes[1]))(_pml_slab(1)))
    assert 1e-4 < np.abs(Rd - Ri).max() < 1e-2


def test_split_pml_reflection_against_a_domain_too_long_to_reach():
    steps = 3000
    short = _pml_slab(steps, nz=1000)
    short.wp2[:] = 0.0
    short.nu[:] = 0.0
    short.src_cell, short.probes = 500, [300, 700]
    off = steps + 50
    long = _pml_slab(steps, nz=1000 + 2 * off)
    long.wp2[:] = 0.0
    long.nu[:] = 0.0
    long.src_cell, long.probes = 500 + off, [300 + off, 700 + off]
    _, s1 = oracle.run1d(short, series=True)
    _, s2 = oracle.run1d(long, series=True)
    peak = np.abs(s2).max()
    assert peak > 0.1
    assert np.abs(s1 - s2).max() <= 2e-3 * peak


def test_planted_unmatched_layer_fails_the_lattice_pin(lattice_rt):
    Rd, Td = lattice_rt
    R, T = _rt(_pml_slab(16000), mutant=10)
    hi = slice(70, None)
    assert max(np.abs(R - Rd)[hi].max(), np.abs(T - Td)[hi].max()) > 1e-5


def test_plasma_inside_the_layer_is_refused():
    s = _pml_slab(10)
    s.wp2[2] = 1e20
    with pytest.raises(ValueError):
        oracle.run1d(s)
