"""GPU path vs the FP64 CPU oracle, through the C ABI (needs a GB300).

Tolerances (normwise relative, ||x_gpu - x_ref||_inf / ||x_ref||_inf per field;
for u the vector field): FP64 storage and arithmetic 1e-12, FP32 1e-5, after
100 steps.  State comparisons (one step from a given state) use the same
normwise measure on the deviations f_i - w_i.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1804_02418_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


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


def vel_err(ux, uy, rx, ry):
    den = np.sqrt(rx * rx + ry * ry).max()
    num = np.sqrt((ux - rx) ** 2 + (uy - ry) ** 2).max()
    return num / (den if den > 0 else 1.0)


def field_errors(g, r):
    return dict(n=rel_err(g[0], r[0]), u=vel_err(g[1], g[2], r[1], r[2]), T=rel_err(g[3], r[3]))


def ragged_sample(tau=0.9, F=(2e-5, -1e-5)):
    """150 x 77: two 128-wide tiles with a ragged tail, walls, three contacts."""
    C = W.Contact
    return W.Sample(150, 77, tau=tau, Fx=F[0], Fy=F[1],
                    contacts=[C(0, 20, 24, u_n=0.01), C(0, 100, 24, u_n=-0.01),
                              C(3, 30, 17, n=1.02, T=0.98)])


def nonequilibrium_state(s, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    lat = lbm.Lattice(s)
    n, ux, uy, T = W.random_fields(s, seed, du=0.05, dn=0.02, dT=0.02)
    post = lbm.init(lat, n, ux, uy, T)
    w = lbm.tables().w[:, None, None]
    return lat, post + amp * w * rng.standard_normal(post.shape)


SAMPLES = {
    "ragged_walls_contacts_force": ragged_sample,
    "periodic_x_channel": lambda: W.Sample(140, 40, periodic_x=True, tau=0.7, Fx=1e-4,
                                           contacts=[W.Contact(1, 10, 30, u_n=0.02)]),
    "doubly_periodic": lambda: W.Sample(133, 31, periodic_x=True, periodic_y=True, tau=1.3,
                                        Fx=-3e-5, Fy=5e-5),
    "minimum_11x11": lambda: W.Sample(11, 11, tau=0.6, contacts=[W.Contact(2, 0, 11, u_n=0.05)]),
}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(SAMPLES))
def test_one_step_from_nonequilibrium_state(rl, prec, name):
    s = SAMPLES[name]()
    lat, post = nonequilibrium_state(s, seed=7)
    ref = lbm.step(lat, post)
    with rl.Solver(s, prec=prec) as sv:
        sv.set_state(np.ascontiguousarray(post))
        sv.step(1)
        got = sv.get_state()
    assert rel_err(got, ref) < (1e-13 if prec == "f64" else 2e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_shear_wave_64_after_100_steps(rl, prec):
    s = W.shear_wave(64, 0.8)
    lat = lbm.Lattice(s)
    fields = W.shear_wave_fields(s)
    post = lbm.run(lat, lbm.init(lat, *fields), 100)
    ref = lbm.macroscopic(lat, post)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0, *[np.ascontiguousarray(f) for f in fields])
        sv.step(100)
        got = sv.moments()
        sv.check()
    e = field_errors(got, ref)
    assert max(e.values()) < TOL[prec], e


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_graphene_sample_256x128_after_100_steps(rl, prec):
    s = W.graphene_sample(nx=256, ny=128, contact_width=16, contact_spacing=64, force=1e-5)
    s.contacts[0].u_n = 1e-3
    s.contacts[1].u_n = -1e-3
    lat = lbm.Lattice(s)
    post = lbm.run(lat, lbm.init(lat, *W.rest_fields(s)), 100)
    ref = lbm.macroscopic(lat, post)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0)
        sv.step(100)
        got = sv.moments()
        sv.check()
    e = field_errors(got, ref)
    assert max(e.values()) < TOL[prec], e


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_random_start_after_100_steps(rl, prec):
    s = ragged_sample()
    lat = lbm.Lattice(s)
    fields = W.random_fields(s, seed=11, du=0.02, dn=0.01, dT=0.01)
    post = lbm.run(lat, lbm.init(lat, *fields), 100)
    ref = lbm.macroscopic(lat, post)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0, *[np.ascontiguousarray(f) for f in fields])
        sv.step(100)
        got = sv.moments()
    e = field_errors(got, ref)
    assert max(e.values()) < TOL[prec], e


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_graphene_sample_one_step_and_three_steps(rl, prec):
    """1024 x 512, walls, two 32-wide contacts 256 apart, F = 1e-6, tau = 1: the
    launch configuration the benchmark times.  After 400 GPU steps from rest
    the state is exported; one more GPU step must equal the oracle's step from
    that state, and three more steps must match in (n, u, T)."""
    s = W.graphene_sample()
    lat = lbm.Lattice(s)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0)
        sv.step(400)
        pre = sv.get_state()
        sv.step(1)
        one = sv.get_state()
        sv.step(2)
        got = sv.moments()
        sv.check()
    ref1 = lbm.step(lat, pre)
    assert rel_err(one, ref1) < (1e-13 if prec == "f64" else 2e-6)
    ref3 = lbm.macroscopic(lat, lbm.run(lat, ref1, 2))
    e = field_errors(got, ref3)
    assert max(e.values()) < TOL[prec], e


def test_init_then_moments_matches_oracle(rl):
    s = ragged_sample()
    lat = lbm.Lattice(s)
    fields = W.random_fields(s, seed=5, du=0.3, dn=0.2, dT=0.2)
    ref = lbm.macroscopic(lat, lbm.init(lat, *fields))
    with rl.Solver(s, prec="f64") as sv:
        sv.init(0, *[np.ascontiguousarray(f) for f in fields])
        got = sv.moments()
    e = field_errors(got, ref)
    assert max(e.values()) < 1e-13, e


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_matches_oracle(rl, prec):
    s = ragged_sample()
    lat = lbm.Lattice(s)
    post = lbm.run(lat, lbm.init(lat, *W.rest_fields(s)), 18)
    ua = lbm.macroscopic(lat, post)[1:3]
    post = lbm.step(lat, post)
    ub = lbm.macroscopic(lat, post)[1:3]
    ref = lbm.residual(ua, ub)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0)
        r = sv.step(20, residual=True)
    assert abs(r - ref) < (1e-10 if prec == "f64" else 1e-4) * ref, (r, ref)


def test_checkpoint_restart_is_bitwise(rl):
    s = ragged_sample()
    with rl.Solver(s, prec="f32") as a:
        a.init(0)
        a.step(30)
        saved = a.get_state()
        a.step(20)
        straight = a.get_state()
    with rl.Solver(s, prec="f32") as b:
        b.set_state(saved)
        b.step(20)
        resumed = b.get_state()
    assert np.array_equal(straight, resumed)


def test_borrowed_and_owned_workspace_agree_bitwise(rl):
    s = ragged_sample()
    out = []
    for ws in ("torch", None):
        with rl.Solver(s, prec="f64", workspace=ws) as sv:
            sv.init(0)
            sv.step(25)
            out.append(sv.get_state())
    assert np.array_equal(out[0], out[1])


def test_unphysical_init_sets_error_word(rl):
    s = W.shear_wave(16)
    n, ux, uy, T = W.rest_fields(s)
    ux = ux.copy()
    ux[3, 4] = 1.5                      # |u| >= 1: no equilibrium exists
    with rl.Solver(s, prec="f64") as sv:
        sv.init(0, n, ux, uy, T)
        with pytest.raises(rl.RlbmError) as ei:
            sv.check()
        assert ei.value.code == -4
        sv.check()                      # flag cleared by the previous check


def test_step_before_init_is_rejected(rl):
    with rl.Solver(W.shear_wave(16), prec="f32") as sv:
        with pytest.raises(rl.RlbmError) as ei:
            sv.step(1)
        assert ei.value.code == -6


def test_zero_steps_is_a_no_op(rl):
    s = ragged_sample()
    with rl.Solver(s, prec="f64") as sv:
        sv.init(0)
        sv.step(3)
        a = sv.get_state()
        sv.step(0)
        b = sv.get_state()
    assert np.array_equal(a, b)


def _window(s, fields, x0, y0, w=64):
    """The w x w window of sample s at (x0, y0) as a sample of its own: the
    window's edges that are edges of s keep their walls and contacts; its
    other edges are artificial walls, more than 10 sites from every site
    compared (one step and the moments' pull reach 10 sites)."""
    contacts = []
    for c in s.contacts:
        # a contact on the lower edge, clipped to the window (its ghost values
        # are the same along it)
        lo, hi = max(c.x0, x0), min(c.x0 + c.length, x0 + w)
        if c.edge == 0 and y0 == 0 and lo < hi:
            contacts.append(W.Contact(0, lo - x0, hi - lo, u_n=c.u_n, n=c.n, T=c.T))
    ws = W.Sample(w, w, tau=s.tau, Fx=s.Fx, Fy=s.Fy, contacts=contacts)
    sub = [np.ascontiguousarray(f[y0:y0 + w, x0:x0 + w]) for f in fields]
    ylo = 0 if y0 == 0 else 10
    yhi = w if y0 + w == s.ny else w - 10
    xlo = 0 if x0 == 0 else 10
    xhi = w if x0 + w == s.nx else w - 10
    return ws, sub, (slice(ylo, yhi), slice(xlo, xhi))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_4096x2048_sample_one_step_in_windows(rl, prec):
    """The 4096 x 2048 graphene sample (walls, contacts 32 wide 256 apart,
    F = 1e-6), random fields, one step in the autotuned launch shape; n, u, T
    compared with the oracle run on 64 x 64 windows (interior, the lower
    wall, both contacts, a corner) that contain every site those values
    depend on."""
    s = W.graphene_sample(nx=4096, ny=2048)
    fields = [np.ascontiguousarray(f) for f in W.random_fields(s, 9, du=0.02, dn=0.01, dT=0.01)]
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0, *fields)
        sv.autotune()
        sv.init(0, *fields)
        sv.step(1)
        got = sv.moments()
        sv.check()
    c0, c1 = s.contacts[0].x0, s.contacts[1].x0
    windows = [(1000, 1000), (500, 0), (c0 - 16, 0), (c1 - 16, 0), (c0 + 10, 0),
               (s.nx - 64, s.ny - 64), (0, 0)]
    worst = {}
    for x0, y0 in windows:
        ws, sub, (ys, xs) = _window(s, fields, x0, y0)
        lat = lbm.Lattice(ws)
        ref = lbm.macroscopic(lat, lbm.run(lat, lbm.init(lat, *sub), 1))
        g = [a[y0:y0 + 64, x0:x0 + 64][ys, xs] for a in got]
        r = [a[ys, xs] for a in ref]
        e = field_errors(g, r)
        worst[(x0, y0)] = max(e.values())
        assert max(e.values()) < TOL[prec], ((x0, y0), e)
    print(f"4096 x 2048 {prec}: worst window error {max(worst.values()):.2e}")


def test_fp32_state_continues_in_fp64(rl):
    """The FP32-then-FP64 route to steady state: a state exported by an FP32
    context and loaded into an FP64 context is the same state (to FP64
    rounding), and one FP64 step from it equals the oracle's step from it."""
    s = ragged_sample()
    lat = lbm.Lattice(s)
    fields = [np.ascontiguousarray(f) for f in W.random_fields(s, 13, du=0.05, dn=0.02, dT=0.02)]
    with rl.Solver(s, prec="f32") as sv:
        sv.init(0, *fields)
        sv.step(40)
        st32 = sv.get_state()
    with rl.Solver(s, prec="f64") as sv:
        sv.set_state(st32)
        back = sv.get_state()
        sv.step(1)
        one = sv.get_state()
        sv.check()
    assert np.abs(back - st32).max() <= 4e-16 * np.abs(st32).max()
    assert rel_err(one, lbm.step(lat, st32)) < 1e-13
