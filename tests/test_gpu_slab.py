"""A single domain cut into slabs of rows, stepped on the GPU (needs a GB300).

Each slab is a context of its own (parallel.Slab.local: the slab's rows plus
5 halo rows of each neighbour); after every step the halo rows are refreshed
from the neighbours' rows by raw device copies between the contexts
(rlbm_get_rows_raw / rlbm_set_rows_raw; parallel.exchange_in_process).  All
slabs run in this one process on one GPU, one after another: no kernel waits
for another.  The slabs' own rows equal the single-domain run bit for bit.
(Between GPUs the same rows travel by NCCL point-to-point sends,
parallel.exchange_device: unmeasured on hardware, every box here has one
GPU; the exchange logic itself is tested on CPU ranks in test_slab_cpu.)
"""
import numpy as np
import pytest

from paper_1804_02418_gb300 import parallel, workloads as W

pytestmark = pytest.mark.gpu

C = W.Contact
CASES = {
    "walls_contacts_force": lambda: W.Sample(150, 77, tau=0.9, Fx=2e-5, Fy=-1e-5, contacts=[
        C(0, 20, 24, u_n=0.01), C(2, 30, 20, u_n=0.02), C(1, 100, 16, n=1.01)]),
    "periodic_y": lambda: W.Sample(64, 60, periodic_y=True, tau=0.7, Fx=3e-5,
                                   contacts=[C(2, 0, 9, u_n=0.01)]),
}


@pytest.fixture(scope="module")
def rl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, rlbm
    build.build()
    return rlbm


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("case,world", [("walls_contacts_force", 2), ("walls_contacts_force", 3),
                                        ("periodic_y", 2)])
def test_slabs_on_one_gpu_reproduce_the_single_domain_run(rl, prec, case, world):
    s = CASES[case]()
    fields = [np.ascontiguousarray(f) for f in W.random_fields(s, 4, du=0.02, dn=0.01, dT=0.01)]
    nsteps = 20
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0, *fields)
        sv.step(nsteps)
        ref = sv.get_state()
        sv.check()
    slabs = [parallel.Slab(s, r, world) for r in range(world)]
    solvers = [rl.Solver(sl.local, prec=prec) for sl in slabs]
    try:
        for sl, sv in zip(slabs, solvers):
            sv.init(0, *[sl.local_rows(f) for f in fields])
        for _ in range(nsteps):
            for sv in solvers:
                sv.step(1)
            parallel.exchange_in_process(slabs, solvers)
        covered = 0
        for sl, sv in zip(slabs, solvers):
            got = sl.owned(sv.get_state())
            sv.check()
            assert np.array_equal(got, ref[:, sl.y0:sl.y1]), \
                (sl.rank, float(np.abs(got - ref[:, sl.y0:sl.y1]).max()))
            covered += sl.own
        assert covered == s.ny
    finally:
        for sv in solvers:
            sv.close()


def test_raw_rows_round_trip_and_bounds(rl):
    import torch
    s = W.Sample(40, 23, tau=0.8)
    with rl.Solver(s, prec="f32") as a, rl.Solver(s, prec="f32") as b:
        a.init(0, *[np.ascontiguousarray(f) for f in W.random_fields(s, 1)])
        b.init(0)
        nb = a.rows_raw_bytes(23)
        assert nb == 12 * 23 * 64 * 4 * 4          # ldx = 64 for nx = 40
        buf = a.get_rows_raw(0, 23, torch.empty(nb, dtype=torch.uint8, device="cuda"))
        b.set_rows_raw(0, 23, buf)
        assert np.array_equal(a.get_state(), b.get_state())
        with pytest.raises(rl.RlbmError):
            a.get_rows_raw(20, 5, torch.empty(nb, dtype=torch.uint8, device="cuda"))
