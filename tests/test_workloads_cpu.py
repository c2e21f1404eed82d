"""The synthetic input recipes (workloads.py): seeded, and distributed as
stated (no GPU)."""
import numpy as np

from paper_1804_02418_gb300 import workloads as W


def test_ensemble_follows_its_recipe():
    """256 samples, seed 1234 + i: short side U[128, 1024], aspect U[1, 4],
    tau U[0.6, 2.0], contact width U{8..64}, |F| logU[1e-7, 1e-5]; about
    1.0e6 sites per sample, 2.6e8 in all; identical when regenerated."""
    e = W.ensemble(256)
    assert len(e) == 256
    short = np.array([s.ny for s in e])
    aspect = np.array([s.nx / s.ny for s in e])
    tau = np.array([s.tau for s in e])
    cw = np.array([s.contacts[0].length for s in e])
    F = np.array([s.Fx for s in e])
    assert short.min() >= 128 and short.max() <= 1024
    assert aspect.min() >= 1.0 - 1e-9 and aspect.max() <= 4.0 + 1e-2
    assert tau.min() >= 0.6 and tau.max() <= 2.0
    assert cw.min() >= 8 and cw.max() <= 64
    assert F.min() >= 1e-7 and F.max() <= 1e-5
    lf = np.log10(F)
    assert abs(lf.mean() + 6.0) < 0.15                     # log-uniform over two decades
    sites = np.array([s.sites for s in e])
    assert 0.7e6 < sites.mean() < 1.3e6
    assert 2.0e8 < sites.sum() < 3.2e8
    again = W.ensemble(256)
    assert [(s.nx, s.ny, s.tau, s.Fx) for s in again] == [(s.nx, s.ny, s.tau, s.Fx) for s in e]


def test_bench_sample_geometry():
    """1024 x 512, walls, two 32-wide contacts on y = 0 with centres at
    x = 384 and 640, F = 1e-6 along x, tau = 1."""
    s = W.graphene_sample()
    assert (s.nx, s.ny, s.tau, s.Fx, s.Fy) == (1024, 512, 1.0, 1e-6, 0.0)
    assert not s.periodic_x and not s.periodic_y
    centres = [c.x0 + c.length / 2 for c in s.contacts]
    assert centres == [384.0, 640.0]
    assert all(c.edge == 0 and c.length == 32 for c in s.contacts)


def test_random_fields_are_seeded():
    s = W.Sample(40, 30)
    a = W.random_fields(s, 5)
    b = W.random_fields(s, 5)
    c = W.random_fields(s, 6)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[1], c[1])
