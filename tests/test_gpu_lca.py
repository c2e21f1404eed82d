"""Electric force of the local capacitance approximation on the GPU (Sec. 3).

* Parity with the oracle's run_lca (lagged density gradient), normwise on
  n, u, T after 60 steps: FP64 1e-12, FP32 1e-5, walled sample with contacts
  and a uniform force, and a periodic sample.
* A batch mixing samples with and without the force reproduces each sample
  run alone (to the last bits), and CUDA-graph replay changes nothing.
* The paper's C_g sweep (Sec. 3): the steady flow between an injector and a
  collector does not depend on C_g (e^2 / C_g = 0.1, 1e-4, 0: velocity
  within 2 % of the largest), while the density does respond to the electric
  force (its variations shrink visibly at C_g = 10, not at 1e4).
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


C = W.Contact


def walled():
    return W.Sample(96, 48, tau=0.9, Fx=2e-5, inv_cg=0.3,
                    contacts=[C(0, 20, 12, u_n=0.01), C(0, 60, 12, u_n=-0.01)])


def periodic():
    return W.Sample(64, 40, periodic_x=True, periodic_y=True, tau=0.9, inv_cg=0.3)


def fields(s, seed):
    return [np.ascontiguousarray(f) for f in W.random_fields(s, seed, du=0.02, dn=0.005, dT=0.005)]


def normwise(got, ref):
    n, ux, uy, T = got
    rn, rux, ruy, rT = ref
    du = np.sqrt((ux - rux) ** 2 + (uy - ruy) ** 2).max() / np.sqrt(rux ** 2 + ruy ** 2).max()
    return max(np.abs(n - rn).max() / np.abs(rn).max(), du, np.abs(T - rT).max() / np.abs(rT).max())


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("make", [walled, periodic], ids=["walled", "periodic"])
def test_parity_with_the_oracle(rl, prec, tol, make):
    s = make()
    f = fields(s, 11)
    lat = lbm.Lattice(s)
    post, dn = lbm.run_lca(lat, lbm.init(lat, *f), f[0] - 1.0, 60)
    ref = lbm.macroscopic(lat, post)
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0, *f)
        sv.step(60)
        got = sv.moments(0)
        sv.check()
    assert normwise(got, ref) <= tol
    # the force is really acting: the same run without it differs far above tol
    s0 = make()
    s0.inv_cg = 0.0
    lat0 = lbm.Lattice(s0)
    ref0 = lbm.macroscopic(lat0, lbm.run(lat0, lbm.init(lat0, *f), 60))
    assert normwise(ref0, ref) > 1e2 * tol


def test_mixed_batch_and_graph_replay(rl):
    samples = [walled(), W.Sample(80, 33, tau=1.1, Fy=1e-5), periodic()]
    alone = []
    for i, s in enumerate(samples):
        with rl.Solver(s, prec="f32") as sv:
            sv.init(0, *fields(s, 20 + i))
            sv.step(24)
            alone.append(sv.get_state(0))
    for graph_steps in (0, 6):
        with rl.Solver(samples, prec="f32", graph_steps=graph_steps) as sv:
            for i, s in enumerate(samples):
                sv.init(i, *fields(s, 20 + i))
            sv.step(24)
            for i in range(len(samples)):
                a, b = alone[i], sv.get_state(i)
                assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
            sv.check()


def test_set_state_restarts_with_the_restored_density(rl):
    """Checkpoint / restart: the restored context continues with the density
    of the restored state in place of the previous step's (one step of lag),
    so it agrees with the uninterrupted run to within that lag's effect."""
    s = walled()
    f = fields(s, 5)
    with rl.Solver(s, prec="f64") as sv:
        sv.init(0, *f)
        sv.step(300)
        ck = sv.get_state(0)
        sv.step(30)
        full = sv.moments(0)
    with rl.Solver(s, prec="f64") as sv:
        sv.set_state(ck, 0)
        sv.step(30)
        resumed = sv.moments(0)
    err = normwise(resumed, full)
    print("restart vs uninterrupted:", err)
    assert 0 < err < 3e-2


def steady(rl, inv_cg):
    s = W.Sample(192, 64, tau=1.0, inv_cg=inv_cg,
                 contacts=[C(0, 56, 16, u_n=1e-4), C(0, 120, 16, u_n=-1e-4)])
    with rl.Solver(s, prec="f64", graph_steps=50) as sv:
        sv.init(0)
        r = 1.0
        while r > 1e-8 and sv.steps_done < 80000:
            sv.step(500)
            r = sv.step(2, residual=True)
        n, ux, uy, T = sv.moments(0)
        sv.check()
    assert r <= 1e-8, r
    return n, ux, uy


def test_steady_flow_does_not_depend_on_the_capacitance(rl):
    n1, ux1, uy1 = steady(rl, 0.1)      # C_g = 10
    n2, ux2, uy2 = steady(rl, 1e-4)     # C_g = 1e4
    n3, ux3, uy3 = steady(rl, 0.0)      # C_g infinite
    umax = np.sqrt(ux3 ** 2 + uy3 ** 2).max()
    for name, ux, uy in (("C_g = 10", ux1, uy1), ("C_g = 1e4", ux2, uy2)):
        du = np.sqrt((ux - ux3) ** 2 + (uy - uy3) ** 2).max() / umax
        print(f"steady u, {name} vs infinite: max |du| / max |u| = {du:.2e}")
        assert du <= 0.02
    # the density does respond to the electric force (its variations shrink),
    # at C_g = 10 visibly and at C_g = 1e4 hardly
    var = lambda n: (n - n.mean()).std()
    r1, r2 = var(n1) / var(n3), var(n2) / var(n3)
    print(f"density variation ratio vs infinite: C_g = 10 {r1:.4f}, C_g = 1e4 {r2:.6f}")
    assert r1 < 0.99
    assert abs(r2 - 1.0) < 1e-3
