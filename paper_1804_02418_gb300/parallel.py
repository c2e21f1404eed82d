"""Host-side logic for runs over several GPUs (one process per GPU).

The method has no exchange step between independent samples, so an ensemble
is sharded by sample with no data-path collective.  A single coupled domain
can be cut into horizontal slabs (ranges of rows), one per rank: a site's
update pulls populations from at most one hop (5 sites) away, so each slab
keeps HALO = 5 rows of each neighbour's post-collision state beside its own
rows and receives them again after every step (the method's one exchange
step; point-to-point sends of torch.distributed, gloo on the host or NCCL
between GPUs, no multicast).  The remaining collectives are for timing and
reporting (max of the per-rank times, sums of the per-rank work).
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable, List, Optional, Sequence

from . import workloads

HALO = workloads.HOP_RADIUS      # rows a site's pull can reach above or below it


def shard_samples(sites: Sequence[int], rank: int, world: int) -> List[int]:
    """Indices of the samples rank `rank` owns: greedy largest-first
    assignment to the least-loaded rank (deterministic, balanced in sites)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world")
    order = sorted(range(len(sites)), key=lambda i: (-sites[i], i))
    load = [0] * world
    owner = [0] * len(sites)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += sites[i]
    return [i for i in range(len(sites)) if owner[i] == rank]


def max_over_ranks(x: float, device="cpu") -> float:
    """Maximum of a per-rank scalar (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_per_rank: float, device="cpu") -> float:
    """Whole-job throughput: sum of every rank's units over the slowest rank's time."""
    units = sum_over_ranks(units_per_rank, device)
    t = max_over_ranks(seconds_per_rank, device)
    return units / t if t > 0 else float("inf")


# ---------------------------------------------------------------------------
# Single-domain slab decomposition (rows), width-5 halo exchange
# ---------------------------------------------------------------------------

def slab_rows(ny: int, world: int) -> List[tuple]:
    """Owned row ranges [y0, y1) of `world` slabs, as even as possible."""
    if world < 1 or ny < world * HALO:
        raise ValueError("every slab must own at least HALO rows")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((y, y + n))
        y += n
    return out


class Slab:
    """Rank `rank`'s slab of `sample` (a workloads.Sample) cut into `world`
    slabs of rows.  Local rows: `lo` halo rows (the rows just below its own,
    owned by rank `down`), its own rows y0 .. y1 - 1, `hi` halo rows (owned by
    `up`).  `local` is the sample the rank steps: the slab's rows with the
    sample's walls, contacts and force; a cut is not periodic, and the pulls
    that cross a local edge at a cut belong to halo rows only, whose results
    the next exchange overwrites.  On a periodic y axis the first and last
    slabs are neighbours."""

    def __init__(self, sample, rank: int, world: int):
        self.rank, self.world = rank, world
        self.y0, self.y1 = slab_rows(sample.ny, world)[rank]
        per = bool(sample.periodic_y)
        cut_below = world > 1 and (rank > 0 or per)
        cut_above = world > 1 and (rank < world - 1 or per)
        self.lo = HALO if cut_below else 0
        self.hi = HALO if cut_above else 0
        self.down = (rank - 1) % world if cut_below else None
        self.up = (rank + 1) % world if cut_above else None
        self.own = self.y1 - self.y0
        ny_local = self.own + self.lo + self.hi
        first = self.y0 - self.lo                      # global row of local row 0
        contacts = []
        for c in sample.contacts:
            if c.edge == workloads.EDGE_Y0:
                if not cut_below:
                    contacts.append(c)
            elif c.edge == workloads.EDGE_Y1:
                if not cut_above:
                    contacts.append(c)
            else:                                      # x edges: span along y, clipped
                for shift in ((-sample.ny, 0, sample.ny) if per else (0,)):
                    a = max(c.x0 + shift, first)       # (a periodic axis wraps the span)
                    b = min(c.x0 + c.length + shift, first + ny_local)
                    if a < b:
                        contacts.append(replace(c, x0=a - first, length=b - a))
        if len(contacts) > workloads.MAX_CONTACTS:
            raise ValueError("a slab would hold more contact segments than a sample may")
        self.first = first
        self.local = replace(sample, ny=ny_local, periodic_y=per and world == 1,
                             contacts=contacts)

    def local_rows(self, a):
        """Rows of a global array [..., ny, nx] this slab holds (halo included,
        wrapped on a periodic axis)."""
        import numpy as np
        ny = a.shape[-2]
        idx = [(self.first + k) % ny for k in range(self.local.ny)]
        return np.ascontiguousarray(np.take(a, idx, axis=-2))

    def owned(self, a):
        """The slab's own rows of a local array [..., ny_local, nx]."""
        return a[..., self.lo:self.lo + self.own, :]

    def exchange(self, state, group=None):
        """Refreshes the halo rows of `state` (a torch tensor [..., ny_local,
        nx], on the host with gloo or on the GPU with NCCL) with the
        neighbours' own rows.  Messages go down first, then up, so that two
        ranks that are each other's up and down neighbour (two slabs on a
        periodic axis) match them in order."""
        import torch
        import torch.distributed as dist
        ops, fills = [], []
        own_lo, own_hi = self.lo, self.lo + self.own
        if self.down is not None:
            buf = state[..., own_lo:own_lo + HALO, :].contiguous()
            ops.append(dist.P2POp(dist.isend, buf, self.down, group, tag=0))
        if self.up is not None:
            buf = state[..., own_hi - HALO:own_hi, :].contiguous()
            ops.append(dist.P2POp(dist.isend, buf, self.up, group, tag=1))
        if self.up is not None:            # the up neighbour's bottom rows: my top halo
            buf = torch.empty_like(state[..., own_hi:own_hi + HALO, :].contiguous())
            ops.append(dist.P2POp(dist.irecv, buf, self.up, group, tag=0))
            fills.append((own_hi, buf))
        if self.down is not None:          # the down neighbour's top rows: my bottom halo
            buf = torch.empty_like(state[..., 0:HALO, :].contiguous())
            ops.append(dist.P2POp(dist.irecv, buf, self.down, group, tag=1))
            fills.append((0, buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for y, buf in fills:
            state[..., y:y + HALO, :] = buf
        return state


def run_slab(slab: Slab, state, nsteps: int, step: Callable, group=None):
    """nsteps time steps of one slab: `step` maps the local post-collision
    state to the next one (stream + collide of the local sample, by whatever
    computes it), then the halo rows are refreshed from the neighbours.  The
    state's halo rows must be current on entry (as after an initialisation
    from global fields, or an exchange)."""
    for _ in range(nsteps):
        state = step(state)
        slab.exchange(state, group)
    return state


def exchange_device(slab: Slab, solver, group=None):
    """Halo exchange of a slab stepped on the GPU by the library (solver: an
    rlbm.Solver of slab.local, one sample): the slab's own boundary rows are
    read raw from the device state (rlbm_get_rows_raw), sent to the
    neighbours and received from them with point-to-point operations of
    torch.distributed (NCCL), and written raw into the halo rows
    (rlbm_set_rows_raw): the values move bit for bit.  Messages are ordered as
    in Slab.exchange.  The solver's stream is synchronised around the
    exchange."""
    import torch
    import torch.distributed as dist
    nb = solver.rows_raw_bytes(HALO)
    mk = lambda: torch.empty(nb, dtype=torch.uint8, device="cuda")
    own_lo, own_hi = slab.lo, slab.lo + slab.own
    ops, fills = [], []
    if slab.down is not None:
        ops.append(dist.P2POp(dist.isend, solver.get_rows_raw(own_lo, HALO, mk()), slab.down,
                              group, tag=0))
    if slab.up is not None:
        ops.append(dist.P2POp(dist.isend, solver.get_rows_raw(own_hi - HALO, HALO, mk()), slab.up,
                              group, tag=1))
    if slab.up is not None:
        b = mk()
        ops.append(dist.P2POp(dist.irecv, b, slab.up, group, tag=0))
        fills.append((own_hi, b))
    if slab.down is not None:
        b = mk()
        ops.append(dist.P2POp(dist.irecv, b, slab.down, group, tag=1))
        fills.append((0, b))
    torch.cuda.synchronize()
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    torch.cuda.synchronize()
    for y, b in fills:
        solver.set_rows_raw(y, HALO, b)


def exchange_in_process(slabs: Sequence[Slab], solvers):
    """The same exchange for slabs stepped by one process on one GPU (one
    context per slab): device copies between the contexts' states."""
    import torch
    torch.cuda.synchronize()
    for sl, sv in zip(slabs, solvers):
        nb = sv.rows_raw_bytes(HALO)
        if sl.down is not None:      # my own bottom rows -> the down neighbour's top halo
            b = sv.get_rows_raw(sl.lo, HALO, torch.empty(nb, dtype=torch.uint8, device="cuda"))
            torch.cuda.synchronize()
            dn = slabs[sl.down]
            solvers[sl.down].set_rows_raw(dn.lo + dn.own, HALO, b)
        if sl.up is not None:        # my own top rows -> the up neighbour's bottom halo
            b = sv.get_rows_raw(sl.lo + sl.own - HALO, HALO,
                                torch.empty(nb, dtype=torch.uint8, device="cuda"))
            torch.cuda.synchronize()
            solvers[sl.up].set_rows_raw(0, HALO, b)
    torch.cuda.synchronize()
