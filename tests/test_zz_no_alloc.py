"""The allocation-free residual entry point against rlbm_step's residual (GPU).

rlbm_velocity_residual_static serves callers that cannot allocate device
memory when they check convergence; it keeps its partial sums in a fixed
array inside the library.  This file is collected last so that a run which
stops at the first failure has already run every other test.

Both calls below go through the C ABI.  The velocity fields u(t-1), u(t) are
the library's own rlbm_moments outputs after 18 and 19 steps, which are the
fields rlbm_step(20, residual) reduces in its last two launches; the two
results must agree within the residual tolerance of the FP64 parity tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1804_02418_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, rlbm
    build.build()
    return torch, rlbm


def sample():
    C = W.Contact
    return W.Sample(150, 77, tau=0.9, Fx=2e-5, Fy=-1e-5,
                    contacts=[C(0, 20, 24, u_n=0.01), C(0, 100, 24, u_n=-0.01)])


def fields_after(torch, rlbm, s, steps):
    """(ux, uy) device tensors after `steps` steps from rest."""
    with rlbm.Solver(s, prec="f64") as sv:
        sv.init(0)
        sv.step(steps)
        out = [torch.empty((s.ny, s.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        sv.moments(0, out=out)
        torch.cuda.synchronize()
    return out[1], out[2]


def existing_residual(rlbm, s, steps):
    with rlbm.Solver(s, prec="f64") as sv:
        sv.init(0)
        return sv.step(steps, residual=True)


def static_residual(torch, rlbm, uxp, uyp, ux, uy, out):
    lib = rlbm.load_library()
    stream = torch.cuda.current_stream()
    rc = lib.rlbm_velocity_residual_static(
        ctypes.c_void_p(uxp.data_ptr()), ctypes.c_void_p(uyp.data_ptr()),
        ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr()),
        ux.numel(), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.rlbm_last_error(None)
    torch.cuda.synchronize()
    return float(out.item())


def test_static_residual_matches_rlbm_step_on_two_calls_in_a_row(env):
    torch, rlbm = env
    s = sample()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # first call: fields at 18 and 19 steps; second call: 38 and 39 steps
    for steps in (20, 40):
        uxp, uyp = fields_after(torch, rlbm, s, steps - 2)
        ux, uy = fields_after(torch, rlbm, s, steps - 1)
        ref = existing_residual(rlbm, s, steps)
        got = static_residual(torch, rlbm, uxp, uyp, ux, uy, out)
        assert ref > 0
        assert abs(got - ref) <= RTOL * ref, (steps, got, ref)


def torch_residual(torch, uxp, uyp, ux, uy):
    """The same quantity by torch float64 reductions (another summation order)."""
    du2 = ((ux - uxp) ** 2 + (uy - uyp) ** 2).sum()
    u2 = (ux ** 2 + uy ** 2).sum()
    return float(torch.sqrt(du2 / u2).item())


def test_static_residual_large_maximum_then_small_sizes(env):
    """Paths the 150 x 77 case does not reach: more partial blocks than the
    final kernel's threads (strided final loop), the largest accepted size
    (every scratch slot written), and a small call right after a large one
    (slots beyond its own block count must not be read)."""
    torch, rlbm = env
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(7)
    for n in (1_500_001, 8_388_608, 333, 2048, 2049):
        uxp, uyp = (1e-3 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
                    for _ in range(2))
        ux = uxp + 1e-6 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        uy = uyp + 1e-6 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        ref = torch_residual(torch, uxp, uyp, ux, uy)
        got = static_residual(torch, rlbm, uxp, uyp, ux, uy, out)
        assert abs(got - ref) <= 1e-12 * ref, (n, got, ref)
        del uxp, uyp, ux, uy


def test_static_residual_rejects_sizes_beyond_its_scratch(env):
    torch, rlbm = env
    lib = rlbm.load_library()
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(a.data_ptr())
    rc = lib.rlbm_velocity_residual_static(p, p, p, p, 8_388_609, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"8388608" in lib.rlbm_last_error(None)
    rc = lib.rlbm_velocity_residual_static(p, p, p, p, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
