"""Contiguous z-domain decomposition with a halo of T steps (host logic).

A Yee step moves information by one cell per step: E_k^{n+1} depends on H_{k-1/2}, H_{k+1/2} of
the half step, which depend on E_{k-1}, E_k, E_{k+1} of step n (Eqs. 12-14; in 3D, the same along
z plane by plane). So a rank that holds its own cells [lo, hi) plus g cells on each side, all of
them exact at the start of a pass, can advance T <= g - d steps alone and still have every owned
cell exact, where d is the depth of what its window ends do that the global problem does not:
0 for an end cell that is merely held or set by a Mur formula (the error then starts in that one
cell), the layer thickness for an absorbing layer (CPML, the split-field PML: its cells go wrong
in the first step). After the pass the ghost cells are stale; the next pass starts by copying
every ghost cell from the rank that owns it. That is the only exchange: once per T steps, g
cells of every state array across each cut, between neighbouring ranks only.

Everything here is plain host logic over torch.distributed point-to-point calls, so the same code
drives CPU ranks (gloo, host tensors) and GPU ranks (NCCL, device tensors): what a rank's window
holds and how it steps are the caller's (a "stepper" with `arrays()` and `step(n)`).

Index conventions: arrays are stored window-local with the z cell (plane) as the leading axis. A
per-cell array (E, J, CPML memories of E; in 3D every component of a plane) has one entry per
cell of the window; a per-interface array (H_{k+1/2} in 1D) has one per interface, index k for
H_{k+1/2}, and one fewer entries. Probes and the source are given by global cell index.
"""
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

CELL, INTERFACE = 0, 1


@dataclass(frozen=True)
class ZDomain:
    """The cells one rank owns ([lo, hi)) and holds ([wlo, whi): owned plus up to g ghosts a side)."""

    rank: int
    world: int
    nz: int
    lo: int
    hi: int
    wlo: int
    whi: int
    ghost: int
    end_depth: int

    @property
    def n(self) -> int:
        """Window length in cells."""
        return self.whi - self.wlo

    @property
    def left_cut(self) -> bool:
        """The window's left end is a cut (not the global boundary)."""
        return self.wlo > 0

    @property
    def right_cut(self) -> bool:
        return self.whi < self.nz

    def local(self, k: int) -> int:
        return k - self.wlo

    def owns(self, k: int) -> bool:
        return self.lo <= k < self.hi

    def array_range(self, kind: int) -> Tuple[int, int]:
        """Global index range a window array of this kind covers."""
        return self.wlo, self.whi - kind

    def exact_zone(self, k: int) -> bool:
        """Whether global cell k lies in the window outside the layers at its cut ends (where the
        window's own end treatment differs from the global problem from the first step)."""
        if not self.wlo <= k < self.whi:
            return False
        if self.left_cut and k < self.wlo + self.end_depth + 1:
            return False
        if self.right_cut and k > self.whi - 2 - self.end_depth:
            return False
        return True


def plan_z(nz: int, world: int, steps_per_pass: int, end_depth: int = 0) -> List[ZDomain]:
    """Splits nz cells into `world` contiguous owned ranges as equal as possible (the first
    nz % world ranks take one more), with ghost width g = steps_per_pass + end_depth. Every owned
    range must hold at least g + 1 cells, so that each ghost cell has its owner among the two
    neighbours and each cut stays clear of the other cut's ghosts."""
    if world < 1 or nz < 1 or steps_per_pass < 1 or end_depth < 0:
        raise ValueError("plan_z needs nz >= 1, world >= 1, steps_per_pass >= 1, end_depth >= 0")
    g = steps_per_pass + end_depth
    base, extra = divmod(nz, world)
    out = []
    lo = 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        if world > 1 and hi - lo < g + 1:
            raise ValueError(f"rank {r} owns {hi - lo} cells, fewer than the ghost width {g} + 1")
        out.append(ZDomain(r, world, nz, lo, hi, max(0, lo - g), min(nz, hi + g), g, end_depth))
        lo = hi
    return out


def _span(a: Tuple[int, int], b: Tuple[int, int]) -> Tuple[int, int]:
    lo, hi = max(a[0], b[0]), min(a[1], b[1])
    return (lo, hi) if lo < hi else (lo, lo)


def transfers(plan: Sequence[ZDomain], rank: int, kind: int) -> List[Tuple[int, str, Tuple[int, int]]]:
    """The strips of one array kind that `rank` sends to and receives from its neighbours:
    (neighbour, "send" or "recv", global index range). A strip is the part of the sender's owned
    cells inside the receiver's window, limited to what both windows' arrays hold."""
    me = plan[rank]
    out = []
    for nb in (rank - 1, rank + 1):
        if not 0 <= nb < len(plan):
            continue
        other = plan[nb]
        both = _span(me.array_range(kind), other.array_range(kind))
        out.append((nb, "send", _span((me.lo, me.hi), both)))
        out.append((nb, "recv", _span((other.lo, other.hi), both)))
    return out


def halo_exchange(plan: Sequence[ZDomain], rank: int, arrays: Sequence[Tuple[torch.Tensor, int]], group=None):
    """Copies every ghost cell of every array from the rank that owns it. `arrays` are window
    arrays (leading axis = cell or interface, contiguous) with their kind (CELL or INTERFACE).
    Point-to-point only (torch.distributed isend/irecv), all posted before any wait."""
    import torch.distributed as dist

    me = plan[rank]
    reqs, landing = [], []
    for a_idx, (arr, kind) in enumerate(arrays):
        if arr.shape[0] != me.n - kind:
            raise ValueError(f"array {a_idx}: leading size {arr.shape[0]}, the window holds {me.n - kind}")
        for nb, how, (g0, g1) in transfers(plan, rank, kind):
            if g1 <= g0:
                continue
            view = arr[g0 - me.wlo:g1 - me.wlo]
            # tag: the array and the direction of travel (towards larger z or not), so that the
            # two strips a pair of ranks swaps for one array never mix
            upward = (nb > rank) if how == "send" else (nb < rank)
            tag = 2 * a_idx + (1 if upward else 0)
            if how == "send":
                out = view.contiguous()
                landing.append((None, out))  # keeps the send buffer alive until the waits
                reqs.append(dist.isend(out, dst=nb, tag=tag, group=group))
            else:
                buf = torch.empty_like(view)
                reqs.append(dist.irecv(buf, src=nb, tag=tag, group=group))
                landing.append((view, buf))
    for r in reqs:
        r.wait()
    for view, buf in landing:
        if view is not None:
            view.copy_(buf)


def run_passes(plan: Sequence[ZDomain], rank: int, stepper, n_steps: int, steps_per_pass: int, group=None) -> int:
    """Advances a rank's window by n_steps in passes of at most steps_per_pass steps, each
    starting with a halo exchange. Returns the number of passes."""
    if steps_per_pass > plan[rank].ghost - plan[rank].end_depth:
        raise ValueError("steps_per_pass exceeds the ghost width less the end depth")
    done, passes = 0, 0
    while done < n_steps:
        halo_exchange(plan, rank, stepper.arrays(), group)
        k = min(steps_per_pass, n_steps - done)
        stepper.step(k)
        done += k
        passes += 1
    return passes


def owned_probes(dom: ZDomain, probes: Sequence[int]) -> List[Tuple[int, int]]:
    """(index in the global probe list, window-local cell) of the probes this rank owns."""
    return [(p, dom.local(k)) for p, k in enumerate(probes) if dom.owns(k)]


def window_source(dom: ZDomain, src_cell: int) -> Optional[int]:
    """Window-local source cell if the window must apply the source (it lies in the window outside
    the layers of its cut ends), else None: the window then runs without a source."""
    return dom.local(src_cell) if dom.exact_zone(src_cell) else None


def sum_spectra(X: torch.Tensor, group=None) -> torch.Tensor:
    """Every rank's spectra rows (zero where it owns no probe) summed over the ranks: each probe
    has one owner, so the sum is that owner's value exactly."""
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return X
    Y = X.clone()
    dist.all_reduce(Y, op=dist.ReduceOp.SUM, group=group)
    return Y
