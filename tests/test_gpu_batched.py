"""Batched ensembles: one launch per step over samples of uneven size (GPU).

The batched kernel runs the same per-site arithmetic as the single-sample
kernel, so a batch whose samples all carry a force must reproduce every
sample run alone bit for bit, for every launch shape the autotuner may pick
(including the persistent kernel whose pulls are staged in shared memory by
bulk asynchronous copies) and with CUDA-graph replay, to the last bits (the
bounds and why they are not all zero are stated at SHAPE_TOL).  A force-free sample inside a forced batch runs
the forced instantiation (zero force adds exact zeros, but the compiler's
multiply-add contraction may differ), so it is compared within the parity
tolerances instead.  A small batch is also checked against the FP64 oracle.
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


def uneven_batch():
    C = W.Contact
    return [
        W.Sample(150, 77, tau=0.9, Fx=2e-5, Fy=-1e-5,
                 contacts=[C(0, 20, 24, u_n=0.01), C(0, 100, 24, u_n=-0.01)]),
        W.Sample(64, 64, periodic_x=True, periodic_y=True, tau=0.8, Fx=3e-5),
        W.Sample(300, 41, tau=1.7, Fx=-1e-5, contacts=[C(1, 10, 30, n=1.01)]),
        W.Sample(11, 11, tau=0.6, Fy=1e-5),
        W.Sample(97, 130, periodic_x=True, tau=1.2, Fy=2e-5, contacts=[C(0, 5, 40, u_n=0.02)]),
        W.Sample(257, 33, tau=2.0, Fx=1e-6, contacts=[C(2, 3, 20, u_n=0.01), C(3, 3, 20)]),
    ]


def fields(s, seed):
    return [np.ascontiguousarray(f) for f in W.random_fields(s, seed, du=0.02, dn=0.01, dT=0.01)]


def run_batch(rl, samples, prec, steps, graph_steps=0, tune=False, shape=None):
    with rl.Solver(samples, prec=prec, graph_steps=graph_steps) as sv:
        for i, s in enumerate(samples):
            sv.init(i, *fields(s, 100 + i))
        if shape is not None:
            sv.set_launch_shape(*shape)
        shape = sv.autotune() if tune else shape
        sv.step(steps)
        out = [sv.get_state(i) for i in range(len(samples))]
        sv.check()
    return out, shape


def run_alone(rl, samples, prec, steps):
    out = []
    for i, s in enumerate(samples):
        with rl.Solver(s, prec=prec) as sv:
            sv.init(0, *fields(s, 100 + i))
            sv.step(steps)
            out.append(sv.get_state(0))
    return out


@pytest.mark.parametrize("prec", ["f32", "f64", "f16dev"])
def test_batch_equals_samples_run_alone_bitwise(rl, prec):
    samples = uneven_batch()
    alone = run_alone(rl, samples, prec, 23)
    batch, _ = run_batch(rl, samples, prec, 23)
    for a, b in zip(alone, batch):
        assert np.array_equal(a, b)


# (sites per block, blocks, staged pulls): one block per tile, persistent
# grids far smaller than the tile list (each block walks many tiles, so the
# two staging buffers alternate many times), and one full wave of 4 blocks / SM
SHAPES = [(64, 0, 0), (256, 0, 0),
          (128, 0, 1), (64, 7, 1), (128, 3, 1), (256, 5, 1), (128, 608, 1)]

# Every kernel runs the same per-site arithmetic, but the code generator
# contracts multiply-adds per kernel (register budgets differ), so results may
# differ in the last bits: measured after 17 steps, FP64 1.4e-15 relative;
# 16-bit storage 4e-4 of the largest deviation (a few values rounded to the
# neighbouring 16-bit code); FP32 bit for bit.
SHAPE_TOL = {"f64": 1e-14, "f32": 0.0, "f16dev": 2e-3, "bf16dev": 2e-2}


@pytest.mark.parametrize("prec", ["f32", "f64", "f16dev", "bf16dev"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda v: "x".join(map(str, v)))
def test_every_launch_shape_equals_samples_run_alone(rl, prec, shape):
    samples = uneven_batch()
    alone = run_alone(rl, samples, prec, 17)
    batch, _ = run_batch(rl, samples, prec, 17, shape=shape)
    for a, b in zip(alone, batch):
        assert np.abs(a - b).max() <= SHAPE_TOL[prec] * np.abs(a).max()


def test_staged_shape_on_the_benchmark_sample_equals_single_sample_kernel(rl):
    s = W.graphene_sample()
    out = []
    for shape in ((0, 0, 0), (128, 608, 1), (64, 1216, 1), (128, 0, 0)):
        with rl.Solver(s, prec="f32", graph_steps=4) as sv:
            sv.init(0, *fields(s, 5))
            sv.set_launch_shape(*shape)
            sv.step(12)
            out.append(sv.get_state(0))
            sv.check()
    for o in out[1:]:
        assert np.array_equal(out[0], o)


def test_invalid_launch_shapes_are_rejected(rl):
    with rl.Solver(uneven_batch()[:2], prec="f32") as sv:
        for bad in ((32, 0, 0), (0, 5, 0), (0, 0, 1), (128, -1, 0), (128, 0, 2)):
            with pytest.raises(rl.RlbmError):
                sv.set_launch_shape(*bad)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f64", 1e-13)])
def test_force_free_sample_in_a_forced_batch(rl, prec, tol):
    samples = uneven_batch()[:3] + [W.Sample(40, 30, tau=0.7)]
    alone = run_alone(rl, samples, prec, 23)
    batch, _ = run_batch(rl, samples, prec, 23)
    for a, b in zip(alone[:3], batch[:3]):
        assert np.array_equal(a, b)
    assert np.abs(alone[3] - batch[3]).max() <= tol * np.abs(alone[3]).max()


def test_autotuned_shape_and_graph_replay_are_bitwise_identical(rl):
    samples = uneven_batch()
    ref, _ = run_batch(rl, samples, "f32", 26)
    tuned, shape = run_batch(rl, samples, "f32", 26, graph_steps=8, tune=True)
    assert shape[0] in (64, 128, 256)
    for a, b in zip(ref, tuned):
        assert np.array_equal(a, b)


def test_single_sample_graph_replay_is_bitwise_identical(rl):
    s = uneven_batch()[0]
    out = []
    for g in (0, 6):
        with rl.Solver(s, prec="f32", graph_steps=g) as sv:
            sv.init(0, *fields(s, 1))
            sv.step(25)
            out.append(sv.get_state(0))
    assert np.array_equal(out[0], out[1])


def test_batch_matches_oracle_per_sample(rl):
    samples = uneven_batch()[:4]
    with rl.Solver(samples, prec="f64") as sv:
        for i, s in enumerate(samples):
            sv.init(i, *fields(s, 100 + i))
        sv.step(30)
        got = [sv.moments(i) for i in range(len(samples))]
    for i, s in enumerate(samples):
        lat = lbm.Lattice(s)
        ref = lbm.macroscopic(lat, lbm.run(lat, lbm.init(lat, *fields(s, 100 + i)), 30))
        for g, r in zip(got[i], ref):
            assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("shape", [None, (128, 3, 1)], ids=["default", "staged"])
def test_per_sample_residuals(rl, shape):
    samples = uneven_batch()
    with rl.Solver(samples, prec="f64") as sv:
        for i, s in enumerate(samples):
            sv.init(i, *fields(s, 100 + i))
        if shape:
            sv.set_launch_shape(*shape)
        total = sv.step(12, residual=True)
        per = sv.sample_residuals()
    alone = []
    for i, s in enumerate(samples):
        with rl.Solver(s, prec="f64") as sv:
            sv.init(0, *fields(s, 100 + i))
            alone.append(sv.step(12, residual=True))
    assert np.allclose(per, alone, rtol=1e-12)
    assert min(per) <= total <= max(per)


@pytest.mark.parametrize("prec", ["f32", "f16dev"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda v: "x".join(map(str, v)))
def test_residual_steps_in_every_launch_shape(rl, prec, shape):
    """The residual-reducing launches (static reduction scratch beside the
    parking area: 48 KiB + 512 B with 256-site blocks) run in every shape and
    give each sample's residual of a run alone."""
    samples = uneven_batch()
    with rl.Solver(samples, prec=prec) as sv:
        for i, s in enumerate(samples):
            sv.init(i, *fields(s, 100 + i))
        sv.set_launch_shape(*shape)
        sv.step(12, residual=True)
        per = sv.sample_residuals()
    alone = []
    for i, s in enumerate(samples):
        with rl.Solver(s, prec=prec) as sv:
            sv.init(0, *fields(s, 100 + i))
            alone.append(sv.step(12, residual=True))
    tol = 1e-12 if prec == "f32" else 1e-2
    assert np.allclose(per, alone, rtol=tol), (per, alone)


def test_autotune_cache_round_trip(rl, tmp_path):
    samples = uneven_batch()[:3]
    import json
    cache = str(tmp_path / "tune.json")
    with rl.Solver(samples, prec="f32", tune_cache=cache) as sv:
        for i, s in enumerate(samples):
            sv.init(i)
        first = sv.autotune()
    d = json.load(open(cache))
    assert len(d) == 1
    (entry,) = d.values()
    assert (entry["bx"], entry["grid"], entry["staged"]) == tuple(first)
    with rl.Solver(samples, prec="f32", tune_cache=cache) as sv:
        for i, s in enumerate(samples):
            sv.init(i)
        assert sv.autotune() == first
    assert json.load(open(cache)) == d
    # a second workload adds its own entry
    with rl.Solver(samples[:1], prec="f32", tune_cache=cache) as sv:
        sv.init(0)
        sv.autotune()
    assert len(json.load(open(cache))) == 2
