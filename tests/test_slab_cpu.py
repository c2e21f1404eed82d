"""Single-domain slab decomposition (parallel.Slab) on CPU ranks.

One sample is cut into slabs of rows, one per rank; each rank steps its slab
plus HALO = 5 rows of each neighbour and refreshes those rows by
point-to-point sends after every step (gloo here; the same calls run on NCCL
between GPUs).  Stepped with the oracle, the ranks' own rows after N steps
equal the single-domain oracle run bit for bit: walls, a contact on the
cut's edge, a contact on an x edge that spans the cut, a force, and a
periodic y axis whose ends are neighbours.  The GPU step over a slab is not
built (every box here has one GPU): unmeasured on hardware.
"""
import os
import socket

import numpy as np
import pytest

from oracle import lbm
from paper_1804_02418_gb300 import parallel, workloads as W

C = W.Contact
CASES = {
    "walls_contacts_force": lambda: W.Sample(36, 31, tau=0.9, Fx=2e-5, Fy=-1e-5, contacts=[
        C(0, 6, 8, u_n=0.01), C(2, 10, 14, u_n=0.02), C(1, 20, 6, n=1.01)]),
    "periodic_y": lambda: W.Sample(24, 33, periodic_y=True, tau=0.7, Fx=3e-5,
                                   contacts=[C(2, 0, 9, u_n=0.01)]),
}


def fields_of(s):
    return W.random_fields(s, 5, du=0.03, dn=0.01, dT=0.01)


def test_slab_rows_partition_and_geometry():
    for ny, world in ((31, 1), (31, 2), (33, 3), (50, 4)):
        rows = parallel.slab_rows(ny, world)
        assert rows[0][0] == 0 and rows[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        assert max(b - a for a, b in rows) - min(b - a for a, b in rows) <= 1
    s = CASES["walls_contacts_force"]()
    lo, hi = parallel.Slab(s, 0, 2), parallel.Slab(s, 1, 2)
    assert (lo.lo, lo.hi, hi.lo, hi.hi) == (0, 5, 5, 0)
    assert lo.local.ny == 16 + 5 and hi.local.ny == 15 + 5
    # the y = 0 contact stays with the bottom slab, the y = ny - 1 one with the top
    assert [c.edge for c in lo.local.contacts].count(0) == 1
    assert [c.edge for c in hi.local.contacts].count(1) == 1
    # the x-edge contact (rows 10 .. 23) is clipped to each slab's local rows
    xl = [c for c in lo.local.contacts if c.edge == 2][0]
    xh = [c for c in hi.local.contacts if c.edge == 2][0]
    assert (xl.x0, xl.x0 + xl.length) == (10, 21)
    assert (xh.x0 + hi.first, xh.x0 + xh.length + hi.first) == (11, 24)
    with pytest.raises(ValueError):
        parallel.slab_rows(8, 2)
    one = parallel.Slab(s, 0, 1)
    assert one.local == s and one.down is None and one.up is None


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, case, nsteps, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = CASES[case]()
        slab = parallel.Slab(s, rank, world)
        lat = lbm.Lattice(slab.local)
        local = [slab.local_rows(f) for f in fields_of(s)]
        post = torch.from_numpy(lbm.init(lat, *local))
        step = lambda t: torch.from_numpy(lbm.step(lat, t.numpy()))
        post = parallel.run_slab(slab, post, nsteps, step)
        out.put((rank, slab.y0, slab.y1, np.array(slab.owned(post).numpy())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("walls_contacts_force", 2), ("walls_contacts_force", 3),
                                        ("periodic_y", 2)])
def test_slabs_reproduce_the_single_domain_run_bitwise(case, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    nsteps = 12
    s = CASES[case]()
    lat = lbm.Lattice(s)
    ref = lbm.run(lat, lbm.init(lat, *fields_of(s)), nsteps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, nsteps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = 0
    for rank, y0, y1, own in res:
        assert np.array_equal(own, ref[:, y0:y1]), (rank, np.abs(own - ref[:, y0:y1]).max())
        covered += y1 - y0
    assert covered == s.ny
