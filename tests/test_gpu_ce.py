"""The Chapman-Enskog seed on the GPU (rlbm_init_ce) against the oracle's
chapman_enskog_init, through the C ABI (needs a GB300).

Stored states are compared normwise on the deviations f_i - w_i, as the
one-step parity tests do: FP64 1e-13 (a direct evaluation, no time stepping),
FP32 2e-6, FP16-deviation storage 1e-3 (its storage rounding, 2^-11 of the
scaled relative deviation).  100 steps from the seed follow the parity bars
of the time-stepping tests (FP64 1e-12, FP32 1e-5 on n, u, T).
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1804_02418_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, rlbm
    build.build()
    return rlbm


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def smooth_fields(s, seed, amp=1.0):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(s.ny), np.arange(s.nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 4)
    n = 1 + amp * 0.02 * np.sin(2 * np.pi * x / s.nx + ph[0]) * np.cos(2 * np.pi * y / s.ny)
    ux = amp * 0.03 * np.sin(2 * np.pi * y / s.ny + ph[1])
    uy = amp * 0.02 * np.cos(2 * np.pi * x / s.nx + ph[2])
    T = 1 + amp * 0.01 * np.cos(2 * np.pi * (x / s.nx + y / s.ny) + ph[3])
    return [np.ascontiguousarray(a) for a in (n, ux, uy, T)]


SAMPLES = {
    "ragged_walls_contacts": lambda: W.Sample(150, 77, tau=0.9, Fx=2e-5, contacts=[
        W.Contact(0, 20, 24, u_n=0.01), W.Contact(3, 30, 17, n=1.02)]),
    "periodic_x_channel": lambda: W.Sample(140, 40, periodic_x=True, tau=0.7),
    "doubly_periodic": lambda: W.Sample(133, 31, periodic_x=True, periodic_y=True, tau=1.3),
    "minimum_11x11": lambda: W.Sample(11, 11, tau=0.6),
}
STATE_TOL = {"f64": 1e-13, "f32": 2e-6, "f16dev": 1e-3}


@pytest.mark.parametrize("prec", list(STATE_TOL))
@pytest.mark.parametrize("name", list(SAMPLES))
def test_seed_state_matches_oracle(rl, prec, name):
    s = SAMPLES[name]()
    lat = lbm.Lattice(s)
    fields = smooth_fields(s, 11)
    ref = lbm.chapman_enskog_init(lat, *fields)
    with rl.Solver(s, prec=prec) as sv:
        sv.init_ce(0, *fields)
        got = sv.get_state()
        sv.check()
    # the seed differs from f^eq (the test is not passed by a plain init)
    assert rel_err(lbm.init(lat, *fields), ref) > 1e-3
    assert rel_err(got, ref) < STATE_TOL[prec], rel_err(got, ref)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_hundred_steps_from_the_seed(rl, prec, tol):
    s = SAMPLES["ragged_walls_contacts"]()
    lat = lbm.Lattice(s)
    fields = smooth_fields(s, 5)
    ref = lbm.macroscopic(lat, lbm.run(lat, lbm.chapman_enskog_init(lat, *fields), 100))
    with rl.Solver(s, prec=prec) as sv:
        sv.init_ce(0, *fields)
        sv.step(100)
        got = sv.moments()
        sv.check()
    for g, r, nm in zip(got, ref, "n ux uy T".split()):
        e = np.abs(g - r).max() / np.abs(r).max()
        assert e < tol, (nm, e)


def test_seed_from_device_fields_and_rest(rl):
    import torch
    s = SAMPLES["periodic_x_channel"]()
    fields = smooth_fields(s, 2)
    dev = [torch.from_numpy(a).cuda() for a in fields]
    with rl.Solver(s, prec="f64") as sv:
        sv.init_ce(0, *fields)
        host = sv.get_state()
        sv.init_ce(0, *dev)
        torch.cuda.synchronize()
        assert np.array_equal(sv.get_state(), host)
        sv.init_ce(0)                         # no fields: the rest state
        assert np.abs(sv.get_state()).max() == 0.0
