"""The z-domain decomposition (paper_1709_00821_gb300/decomp.py) emulated with CPU ranks: two or
three gloo processes, each running the unmodified FP64 oracle on its window (owned cells plus
ghosts), with a halo exchange every T steps. The owned cells of every rank, and the spectra summed
over the ranks, must equal a single-domain oracle run bit for bit: the per-cell arithmetic does not
depend on where a window starts, so any difference is a decomposition error (a ghost too narrow, a
strip off by one, a probe or source on the wrong rank).

Cases: the paper's slab with Mur ends and a halo of 16 steps; a random medium with CPML ends (the
windows' cut ends carry CPML layers too, so the ghost width adds their depth); the split-field PML
with the Eq. 10 recursion, which carries E^{n-1} across the exchange; 3D with PEC z ends and the
one-plane face exchange every step (T = 1); 3D with z CPML and T = 2. A ghost that leaves out the
CPML depth must break the equality (the check is not vacuous). Not run on hardware: one GPU per
process here."""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_1709_00821_gb300 import decomp as dc
from paper_1709_00821_gb300 import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ------------------------------------------------------------------ problems
def _c1_mur():
    s = wl.c1_plain_slab(steps=3000)
    return s, 16, 0


def _random_medium(nz, seed):
    u = wl.uniform01(seed, 2 * nz)
    wp2 = (2 * np.pi * 40e9 * u[:nz]) ** 2 * (u[:nz] > 0.4)
    nu = 1e11 * u[nz:]
    return wp2, nu


def _cpml_random():
    s = wl.c1_plain_slab(nz=1500, steps=1200)
    s.wp2, s.nu = _random_medium(1500, 0xD1)
    s.bc, s.cpml_cells = "cpml", 8
    s.src_cell, s.probes = 40, [60, 700, 1400]
    return s, 8, 8


def _pml_etd2():
    s = wl.c1_plain_slab(nz=1200, steps=900)
    wp2, nu = _random_medium(1200, 0xD2)
    wp2[:5] = wp2[-5:] = 0.0  # the global PML layers are vacuum
    s.wp2, s.nu = wp2, nu
    s.bc, s.cpml_cells, s.scheme = "pml", 5, wl.SCHEME_ETD2
    s.src_cell, s.probes = 30, [20, 600, 1190]
    return s, 12, 5


def _cpml_too_narrow():
    s, T, _ = _cpml_random()
    return s, T, 0  # leaves the cut ends' CPML depth out of the ghost width


CASES_1D = {"c1_mur": _c1_mur, "cpml_random": _cpml_random, "pml_etd2": _pml_etd2,
            "cpml_too_narrow": _cpml_too_narrow}


def _blob3d(npml):
    nx = ny = 8
    nz = 48
    d = 100e-6
    dt = wl.dt_for_courant(d, 0.5)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = ((i - 3.2) ** 2 + (j - 4.1) ** 2 + (k - 26.0) ** 2) < 12
    mat = np.where(inside, 1 | (1 << 2) | (1 << 4), 0).astype(np.uint8)
    mat[30:33] |= np.uint8(2 << 4)  # a thin layer where only Ez sees the second material
    return wl.Grid3D(nx, ny, nz, d, dt, mat.ravel(), np.array([0.0, (2 * np.pi * 40e9) ** 2, (2 * np.pi * 20e9) ** 2]),
                     np.array([0.0, 2e10, 5e10]), True, npml, False, (0, 0, 0, 0, 0, 0), 12, 4 * dt, 12 * dt,
                     [(2, 3, 9), (5, 5, 27), (1, 6, 40)], np.linspace(5e9, 200e9, 9), 150)


CASES_3D = {"pec_one_plane": (lambda: _blob3d(0), 1, 0), "cpml_z": (lambda: _blob3d(4), 2, 4)}


# ------------------------------------------------------------------ oracle windows
class Oracle1DWindow:
    """A rank's window as a 1D oracle problem: the slab's cells [wlo, whi), the source only where
    the window must apply it, the probes it owns; medium zeroed inside the layers at cut ends
    (the split-field PML takes no plasma; those cells go wrong in the first step anyway)."""

    def __init__(self, slab, dom):
        self.dom = dom
        w = slice(dom.wlo, dom.whi)
        wp2, nu = slab.wp2[w].copy(), slab.nu[w].copy()
        c = slab.cpml_cells if slab.bc in ("cpml", "pml") else 0
        if dom.left_cut:
            wp2[:c], nu[:c] = 0.0, 0.0
        if dom.right_cut and c:
            wp2[-c:], nu[-c:] = 0.0, 0.0
        src = dc.window_source(dom, slab.src_cell)
        self.owned = dc.owned_probes(dom, slab.probes)
        self.slab = wl.Slab1D(dom.n, slab.dz, slab.dt, wp2, nu, src if src is not None else 1, slab.src_tau,
                              slab.src_t0, [k for _, k in self.owned], slab.freq_hz, slab.bc, slab.cpml_cells,
                              slab.steps, slab.src_amp if src is not None else 0.0, slab.scheme)
        self.st = oracle.State1D(self.slab)

    def arrays(self):
        st = self.st
        return [(torch.from_numpy(st.E), dc.CELL), (torch.from_numpy(st.H), dc.INTERFACE),
                (torch.from_numpy(st.J), dc.CELL), (torch.from_numpy(st.psiE), dc.CELL),
                (torch.from_numpy(st.psiH), dc.INTERFACE), (torch.from_numpy(st.Eprev), dc.CELL)]

    def step(self, n):
        oracle.run1d(self.slab, steps=n, state=self.st)


class Oracle3DWindow:
    """A rank's window as a 3D oracle problem: planes [wlo, whi), the sheet source where the window
    must apply it, the probes it owns."""

    def __init__(self, prob, dom):
        self.dom = dom
        plane = prob.nx * prob.ny
        sheet = dc.window_source(dom, prob.sheet_k)
        self.owned = [(p, (i, j, dom.local(k))) for p, (i, j, k) in enumerate(prob.probes) if dom.owns(k)]
        self.prob = wl.Grid3D(prob.nx, prob.ny, dom.n, prob.d, prob.dt, prob.mat[dom.wlo * plane:dom.whi * plane].copy(),
                              prob.mat_wp2, prob.mat_nu, prob.periodic_xy, prob.npml, False, (0, 0, 0, 0, 0, 0),
                              sheet if sheet is not None else -1, prob.src_tau, prob.src_t0,
                              [xyz for _, xyz in self.owned], prob.freq_hz, prob.steps)
        self.st = oracle.State3D(self.prob)

    def arrays(self):
        n = self.dom.n
        out = [(torch.from_numpy(self.st.fields[q].reshape(n, -1)), dc.CELL) for q in range(9)]
        out += [(torch.from_numpy(self.st.psi[q].reshape(n, -1)), dc.CELL) for q in range(12)]
        return out

    def step(self, n):
        oracle.run3d(self.prob, steps=n, state=self.st)


# ------------------------------------------------------------------ ranks
def _worker(rank, world, port, dim, case, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if dim == 1:
            prob, T, depth = CASES_1D[case]()
            plan = dc.plan_z(prob.nz, world, T, depth)
            win = Oracle1DWindow(prob, plan[rank])
            nprobe, steps = len(prob.probes), prob.steps
        else:
            build, T, depth = CASES_3D[case]
            prob = build()
            plan = dc.plan_z(prob.nz, world, T, depth)
            win = Oracle3DWindow(prob, plan[rank])
            nprobe, steps = len(prob.probes), prob.steps
        passes = dc.run_passes(plan, rank, win, steps, T)
        X = torch.zeros(2, nprobe, len(prob.freq_hz), dtype=torch.float64)
        for row, (p, _) in enumerate(win.owned):
            X[0, p] = torch.from_numpy(win.st.X[row].real.copy())
            X[1, p] = torch.from_numpy(win.st.X[row].imag.copy())
        X = dc.sum_spectra(X)
        dom = plan[rank]
        a, b = dom.local(dom.lo), dom.local(dom.hi)
        if dim == 1:
            own = {"E": win.st.E[a:b], "H": win.st.H[a:min(b, dom.n - 1)], "J": win.st.J[a:b]}
        else:
            own = {"F": win.st.fields.reshape(9, dom.n, -1)[:, a:b]}
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), X=X.numpy(), lo=dom.lo, hi=dom.hi, passes=passes, **own)
    finally:
        dist.destroy_process_group()


def _run_ranks(tmp_path, world, dim, case):
    import torch.multiprocessing as mp

    mp.spawn(_worker, args=(world, _free_port(), dim, case, str(tmp_path)), nprocs=world, join=True)
    return [dict(np.load(tmp_path / f"r{r}.npz")) for r in range(world)]


def _compare_1d(parts, ref):
    E = np.full_like(ref.E, np.nan)
    H = np.full_like(ref.H, np.nan)
    J = np.full_like(ref.J, np.nan)
    for p in parts:
        lo, hi = int(p["lo"]), int(p["hi"])
        E[lo:hi], J[lo:hi] = p["E"], p["J"]
        H[lo:lo + len(p["H"])] = p["H"]
    X = parts[0]["X"][0] + 1j * parts[0]["X"][1]
    return (np.array_equal(E, ref.E) and np.array_equal(H, ref.H) and np.array_equal(J, ref.J)
            and np.array_equal(X, ref.X))


# ------------------------------------------------------------------ tests
@pytest.mark.parametrize("case,world", [("c1_mur", 3), ("cpml_random", 2), ("pml_etd2", 3), ("c1_mur", 2)])
def test_1d_decomposition_equals_one_domain_bitwise(tmp_path, case, world):
    prob, T, _ = CASES_1D[case]()
    ref, _ = oracle.run1d(prob)
    parts = _run_ranks(tmp_path, world, 1, case)
    assert all(int(p["passes"]) == -(-prob.steps // T) for p in parts)
    assert _compare_1d(parts, ref)


def test_a_ghost_without_the_cut_layer_depth_breaks_the_equality(tmp_path):
    prob, _, _ = CASES_1D["cpml_too_narrow"]()
    ref, _ = oracle.run1d(prob)
    parts = _run_ranks(tmp_path, 2, 1, "cpml_too_narrow")
    assert not _compare_1d(parts, ref)


@pytest.mark.parametrize("case,world", [("pec_one_plane", 3), ("pec_one_plane", 2), ("cpml_z", 2)])
def test_3d_z_slab_decomposition_equals_one_domain_bitwise(tmp_path, case, world):
    build, T, _ = CASES_3D[case]
    prob = build()
    ref, _ = oracle.run3d(prob)
    parts = _run_ranks(tmp_path, world, 3, case)
    F = np.full((9, prob.nz, prob.nx * prob.ny), np.nan)
    for p in parts:
        F[:, int(p["lo"]):int(p["hi"])] = p["F"]
    assert np.abs(ref.fields).max() > 0
    assert np.array_equal(F.reshape(9, -1), ref.fields)
    X = parts[0]["X"][0] + 1j * parts[0]["X"][1]
    assert np.array_equal(X, ref.X)
    if T == 1:
        assert all(int(p["passes"]) == prob.steps for p in parts)  # one face exchange per step


def test_plan_covers_the_line_once_and_strips_pair_up():
    for nz, world, T, depth in [(2000, 3, 16, 0), (1500, 2, 8, 8), (97, 4, 3, 2), (10, 1, 4, 0)]:
        plan = dc.plan_z(nz, world, T, depth)
        assert plan[0].lo == 0 and plan[-1].hi == nz
        assert all(a.hi == b.lo for a, b in zip(plan, plan[1:]))
        assert max(d.hi - d.lo for d in plan) - min(d.hi - d.lo for d in plan) <= 1
        for d in plan:
            assert d.wlo == max(0, d.lo - T - depth) and d.whi == min(nz, d.hi + T - 0 + depth)
        for kind in (dc.CELL, dc.INTERFACE):
            for r in range(world):
                for nb, how, rng in dc.transfers(plan, r, kind):
                    other = "recv" if how == "send" else "send"
                    match = [x for x in dc.transfers(plan, nb, kind) if x[0] == r and x[1] == other]
                    assert match and match[0][2] == rng
                    if how == "recv":  # every ghost cell the window's array holds arrives
                        me = plan[r]
                        lo, hi = me.array_range(kind)
                        ghosts = set(range(lo, hi)) - set(range(me.lo, me.hi))
                        side = set(range(plan[nb].lo, plan[nb].hi))
                        assert ghosts & side == set(range(*rng))


def test_plan_refuses_ranks_narrower_than_the_ghost():
    with pytest.raises(ValueError):
        dc.plan_z(100, 8, 12, 0)
    with pytest.raises(ValueError):
        dc.plan_z(100, 2, 0, 0)


def test_probe_and_source_ownership():
    plan = dc.plan_z(2000, 3, 16, 4)
    probes = [300, 666, 667, 1700]
    owners = [[p for p, _ in dc.owned_probes(d, probes)] for d in plan]
    assert sorted(sum(owners, [])) == [0, 1, 2, 3] and all(len(set(o)) == len(o) for o in owners)
    # the source at a cut: both windows that hold it outside their cut layers apply it
    src = plan[1].lo
    holders = [d.rank for d in plan if dc.window_source(d, src) is not None]
    assert holders == [0, 1]
    # inside rank 1's left cut layer (its first end_depth + 1 cells) rank 1 does not apply it
    assert dc.window_source(plan[1], plan[1].wlo + 2) is None
    assert dc.window_source(plan[0], plan[1].wlo + 2) is not None
