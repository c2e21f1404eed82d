"""What the learned warm start gains over starting from rest (GPU, small scale).

A small operator is trained in seconds on steady states of small walled
samples produced by the batched solver, then used to seed held-out samples.
Starting from rest the initial velocity error is 100 % by definition; the
trained operator must start well below that and reach a given accuracy of
the steady velocity field in no more steps than the rest start.  (Time to a
per-step residual of 1e-6 is measured by paper_1804_02418_gb300.warmstart at
full size; the slow acoustic tail it is dominated by is not shortened by the
seed, see the design notes.)
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, fno, warmstart
    build.build()
    return torch, fno, warmstart


def test_trained_operator_seeds_closer_and_gets_there_no_later(env):
    torch, fno, ws = env
    samples = ws.dataset_samples(112, 777, w_lo=16, w_hi=28, max_aspect=3.0)
    _, _, fields, _ = ws.converge(samples, "f32", max_steps=20000)
    N = 64
    data = ws.build_dataset(samples, fields, N)
    ntr = 96
    m_tr = data.m[:ntr, ..., None]
    chan = np.sqrt((data.y[:ntr] ** 2 * m_tr).sum((0, 1, 2)) / m_tr.sum()).astype(np.float32)
    chan = np.where(chan > 0, chan, 1.0).astype(np.float32)
    data.y /= chan
    tr = ws.Data(data.x[:ntr], data.y[:ntr], data.m[:ntr])
    cfg = fno.FNOConfig(N=N, C=16, Cq=64, L=3, m1=8, m2=8)
    net, hist, _ = ws.train(tr, cfg, epochs=25, batch=8, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    held, ref = samples[ntr:], fields[ntr:]
    pred = ws.predict_fields(net, held, N, use=("n", "u"), chan=chan)
    err = [np.sqrt(((p[1] - r[1]) ** 2 + (p[2] - r[2]) ** 2).sum() / (r[1] ** 2 + r[2] ** 2).sum())
           for p, r in zip(pred, ref)]
    assert np.median(err) < 0.6, np.median(err)
    _, _, _, dc = ws.converge(held, "f64", ref=ref, check=20, max_steps=400)
    _, _, _, dw = ws.converge(held, "f64", init=pred, ref=ref, check=20, max_steps=400)
    for lvl in (0.3, 0.1):
        cold = np.median(ws.steps_to(dc, lvl, check=20))
        warm = np.median(ws.steps_to(dw, lvl, check=20))
        assert warm <= cold, (lvl, warm, cold)
