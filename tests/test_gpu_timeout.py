"""Failure detection on the GPU: a bounded wait that gives up (needs a GB300).

The staged-pull kernel waits on an mbarrier for the bulk copies of each tile.
With the context's wait limit set to one clock cycle, the first wait of every
block gives up before its copies can land (their latency is hundreds of
cycles): the kernel sets the timeout bit of the device error word, waits with
the default bound for the copies it has issued (so no copy into shared memory
is left in flight), and returns.  rlbm_check reports RLBM_ETIMEOUT, and the
context works again once its state is set anew.  Nothing here faults or
hangs the GPU: every wait is bounded and every copy completes.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["f32", "f16dev"])
def test_wait_gives_up_reports_timeout_and_context_recovers(rl, prec):
    s = W.graphene_sample(nx=256, ny=128, contact_width=16, contact_spacing=64, force=1e-5)
    with rl.Solver(s, prec=prec) as ref:
        ref.init(0)
        ref.set_launch_shape(128, 152, 1)
        ref.step(12)
        want = ref.get_state()
        ref.check()
    with rl.Solver(s, prec=prec) as sv:
        sv.init(0)
        sv.set_launch_shape(128, 152, 1)
        sv.set_wait_limit(1)
        sv.step(2)
        with pytest.raises(rl.RlbmError) as e:
            sv.check()
        assert e.value.code == -5, str(e.value)
        sv.check()                              # the bit was cleared by the report
        # back to the default limit: the same run as the reference, bit for bit
        sv.set_wait_limit(0)
        sv.init(0)
        sv.step(12)
        got = sv.get_state()
        sv.check()
    assert np.array_equal(got, want)
