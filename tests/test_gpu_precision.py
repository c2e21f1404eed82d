"""16-bit deviation storage (FP16 / BF16, FP32 arithmetic) against the FP64
oracle, through the C ABI (needs a GB300).

Bar, derived from the storage format: every step stores each relative
deviation g_i = (f_i - w_i) / w_i rounded to p mantissa bits, a relative
error of at most u_p = 2^-(p+1) (FP16 p = 10: 4.9e-4 with the scale s = 1024
keeping the values normal; BF16 p = 7: 3.9e-3).  The moments are sums of
g_i weighted by w_i p_i, so one step moves n, u and T by O(u_p) of their
deviations; over N steps independent roundings add up like a random walk.
The test allows
    normwise error <= 4 u_p sqrt(N)
(n, u, T normwise as in the FP64 / FP32 parity tests: relative to the
largest value of the field, u as a vector field), and checks that FP16
beats BF16 by at least 4x (BF16 has 3 mantissa bits fewer, less a margin).
Measured on GB300 after 100 steps: u within 1.2e-4 / 2.7e-4 (FP16) and
1.1e-3 / 2.1e-3 (BF16) on the shear wave / the 256 x 128 sample; n and T
within 3e-7 (FP16) and 8e-6 (BF16).
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1804_02418_gb300 import workloads as W

pytestmark = pytest.mark.gpu

UNIT = {"f16dev": 2.0 ** -11, "bf16dev": 2.0 ** -8}


@pytest.fixture(scope="module")
def rl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, rlbm
    build.build()
    return rlbm


def errors(got, ref):
    n, ux, uy, T = got
    rn, rux, ruy, rT = ref
    du = np.sqrt((ux - rux) ** 2 + (uy - ruy) ** 2).max() / np.sqrt(rux ** 2 + ruy ** 2).max()
    dn = np.abs(n - rn).max() / np.abs(rn).max()
    dT = np.abs(T - rT).max() / np.abs(rT).max()
    return {"n": dn, "u": du, "T": dT}


CASES = {
    "shear_wave_64": (lambda: W.shear_wave(64, 0.8), lambda s: W.shear_wave_fields(s)),
    "graphene_256x128_random": (
        lambda: W.graphene_sample(nx=256, ny=128, contact_width=16, contact_spacing=64, force=1e-5),
        lambda s: W.random_fields(s, 4, du=0.02, dn=0.01, dT=0.01)),
}
STEPS = 100


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name, (mk, fl) in CASES.items():
        s = mk()
        f = [np.ascontiguousarray(a) for a in fl(s)]
        lat = lbm.Lattice(s)
        out[name] = (s, f, lbm.macroscopic(lat, lbm.run(lat, lbm.init(lat, *f), STEPS)))
    return out


@pytest.mark.parametrize("case", list(CASES))
def test_16_bit_storage_within_the_rounding_bound(rl, refs, case):
    s, f, ref = refs[case]
    worst = {}
    for prec in ("f16dev", "bf16dev"):
        with rl.Solver(s, prec=prec) as sv:
            sv.init(0, *f)
            sv.step(STEPS)
            got = sv.moments(0)
            sv.check()
        e = errors(got, ref)
        worst[prec] = max(e.values())
        bound = 4 * UNIT[prec] * np.sqrt(STEPS)
        print(f"{case} {prec}: {e} (bound {bound:.2e})")
        assert worst[prec] <= bound, (prec, e)
    assert worst["f16dev"] * 4 <= worst["bf16dev"]
