"""Spectral neural operator kernels vs the FP64 oracle (GPU).

* the GEMMs (FP32 units; BF16 on mma.sync and on tcgen05 with a tensor-memory
  accumulator; every transpose / epilogue / batch-stride mode, ragged tiles)
  equal the FP64 product to their accumulation accuracy, and the two BF16
  back ends agree on the full-size operator's shapes;
* the network in its FP32 mode (FP32 weights, activations, DFT matrices and
  GEMMs): forward output, loss and every parameter gradient equal the
  oracle's (numpy.fft definition) element by element within 1e-5 of the
  tensor's largest entry; sizes cover ragged GEMM tiles, the ragged split-K
  remainder and the 16-byte staging paths;
* the network in its BF16 mode (both tensor-core back ends): element by
  element within n_r 2^-8 of the tensor's largest entry, n_r the number of
  BF16 roundings on the longest path to that tensor (each rounding moves a
  value by at most 2^-8 of itself; the network's layers are contractions of
  their inputs' scale at these initialisations).
"""
import numpy as np
import pytest

from oracle import fno as ofno

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02418_gb300 import build, fno
    build.build()
    return torch, fno


def bf16_round(a):
    import torch
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def f32_round(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("impl", ["mma", "tc", "f32"])
@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K,batch", [(70, 45, 37, 3), (128, 64, 96, 1), (5, 300, 64, 2),
                                         (257, 129, 333, 2), (1, 1, 1, 1)])
def test_gemm_bf16_matches_fp64(env, impl, tA, tB, M, N, K, batch):
    torch, fno = env
    f32 = impl == "f32"
    net = fno.FNO(fno.FNOConfig(N=8, C=8, Cq=8, L=1, m1=2, m2=2), batch=1,
                  gemm_impl="tc" if f32 else impl, act="f32" if f32 else "bf16")
    rng = np.random.default_rng(M + N + K + 7 * tA + 3 * tB)
    rnd = f32_round if f32 else bf16_round
    A = rnd(rng.standard_normal((batch, K, M) if tA else (batch, M, K)))
    B = rnd(rng.standard_normal((batch, N, K) if tB else (batch, K, N)))
    bias = rng.standard_normal(N)
    C0 = rng.standard_normal((batch, M, N))
    op = torch.float32 if f32 else torch.bfloat16
    At = torch.tensor(A, dtype=op, device="cuda")
    Bt = torch.tensor(B, dtype=op, device="cuda")
    Ct = torch.tensor(C0, dtype=torch.float32, device="cuda")
    bt = torch.tensor(bias, dtype=torch.float32, device="cuda")
    Dt = torch.empty((batch, M, N), dtype=op, device="cuda")
    net.gemm(At, Bt, M, N, K, lda=M if tA else K, ldb=K if tB else N, transA=tA, transB=tB,
             C=Ct, ldc=N, D=Dt, bias=bt, beta=0.5, epi=fno.EPI_GELU, batch=batch,
             sA=M * K, sB=K * N, sC=M * N, alpha=2.0)
    torch.cuda.synchronize()
    opA = np.transpose(A, (0, 2, 1)) if tA else A
    opB = np.transpose(B, (0, 2, 1)) if tB else B
    ref = 2.0 * opA @ opB + 0.5 * C0 + bias
    got = Ct.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * (np.abs(opA) @ np.abs(opB)).max() * 2 + 1e-5
    g = ofno.gelu(ref)
    dtol = 1e-5 * (np.abs(opA) @ np.abs(opB)).max() * 2 + 1e-5 if f32 else 1e-2 * max(1.0, np.abs(g).max())
    assert np.abs(Dt.float().cpu().numpy() - g).max() <= dtol
    # split-K atomic accumulation over the batch into one output
    Ca = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    net.gemm(At, Bt, M, N, K, lda=M if tA else K, ldb=K if tB else N, transA=tA, transB=tB,
             C=Ca, ldc=N, epi=fno.EPI_ATOMIC, batch=batch, sA=M * K, sB=K * N, sC=0)
    torch.cuda.synchronize()
    assert np.abs(Ca.cpu().numpy() - (opA @ opB).sum(0)).max() <= 1e-4 * batch * (np.abs(opA) @ np.abs(opB)).max()
    assert tc_flag(fno) == 0


def tc_flag(fno):
    import ctypes
    f = ctypes.c_int(-1)
    assert fno._lib().rlbm_gemm_tc_error(ctypes.byref(f)) == 0
    return f.value


def test_tcgen05_and_mma_agree_on_the_operator_shapes(env):
    """The spectral-layer shapes of the full-size operator (N 256, C 32,
    m1 = m2 = 16, batch 8): the two back ends agree to FP32 accumulation."""
    torch, fno = env
    rng = np.random.default_rng(11)
    N, C, m2, B = 256, 32, 16, 8
    cases = [  # (M, N, K, batch, lda, ldb): y-DFT, x-DFT, pointwise W
        (2 * m2, C, N, B * N, N, C),
        (64, m2 * C, 2 * N, B, 2 * N, m2 * C),
        (B * N * N, C, C, 1, C, C),
    ]
    for M, Nn, K, batch, lda, ldb in cases:
        A = torch.tensor(rng.standard_normal((M, K)), dtype=torch.bfloat16, device="cuda")
        Bm = torch.tensor(rng.standard_normal((batch, K, Nn)), dtype=torch.bfloat16, device="cuda")
        outs = []
        for impl in ("mma", "tc"):
            net = fno.FNO(fno.FNOConfig(N=8, C=8, Cq=8, L=1, m1=2, m2=2), batch=1, gemm_impl=impl)
            Cm = torch.empty((batch, M, Nn), dtype=torch.float32, device="cuda")
            net.gemm(A, Bm, M, Nn, K, lda=lda, ldb=ldb, C=Cm, ldc=Nn, batch=batch, sA=0,
                     sB=K * Nn, sC=M * Nn)
            outs.append(Cm)
        torch.cuda.synchronize()
        scale = float((A.float().abs() @ Bm[0].float().abs()).max())
        assert float((outs[0] - outs[1]).abs().max()) <= 2e-6 * scale * max(1.0, K / 64)
    assert tc_flag(fno) == 0


def run_gpu_network(torch, fno, cfg, B, impl, act, seed):
    """GPU forward, loss and backward; returns (y, loss, grads, params, x, t, m)."""
    net = fno.FNO(cfg, batch=B, seed=seed, gemm_impl=impl, act=act)
    rng = np.random.default_rng(seed + 1)
    rnd = f32_round if act == "f32" else bf16_round
    x = rnd(rng.standard_normal((B, cfg.N, cfg.N, cfg.cin)))
    t = rng.standard_normal((B, cfg.N, cfg.N, cfg.cout))
    m = (rng.uniform(size=(B, cfg.N, cfg.N)) < 0.8).astype(float)
    rows = B * cfg.N * cfg.N
    xt = torch.tensor(x.reshape(rows, cfg.cin),
                      dtype=torch.float32 if act == "f32" else torch.bfloat16, device="cuda")
    tt = torch.tensor(t.reshape(rows, cfg.cout), dtype=torch.float32, device="cuda")
    mt = torch.tensor(m.reshape(rows), dtype=torch.float32, device="cuda")
    y = net.forward(xt).cpu().numpy().reshape(B, cfg.N, cfg.N, cfg.cout)
    loss = float(net.loss(tt, mt))
    net.backward()
    torch.cuda.synchronize()
    grads = {n: net.get(n, "grad").cpu().numpy().astype(np.float64) for n in net.offsets}
    grads["R"] = grads["R"][..., 0] + 1j * grads["R"][..., 1]
    pg = net.params_numpy()
    # the oracle takes the weights the GPU GEMMs use (BF16-rounded in BF16 mode)
    wr = (lambda v: v) if act == "f32" else bf16_round
    p = {k: (wr(v) if k in ("P", "W", "Q1", "Q2") else v) for k, v in pg.items()}
    p["R"] = pg["R"][..., 0] + 1j * pg["R"][..., 1]
    return y, loss, grads, p, x, t, m


def oracle_network(cfg, p, x, t, m):
    o = ofno.Oracle(cfg.N, cfg.m1, cfg.m2)
    yo, cache = o.forward(p, x)
    lo, dyo = o.loss(yo, t, m)
    return yo, lo, o.backward(p, cache, dyo)


def elementwise_ok(got, ref, tol):
    """max_e |got_e - ref_e| <= tol * max_e |ref_e| (complex: modulus)."""
    return float(np.abs(got - ref).max()), float(tol * np.abs(ref).max())


# N 20, B 3: 1,200 rows = two 512-row split-K chunks + a ragged 176; C 12, Cq 20,
# 2 m2 = 10: ragged GEMM tiles everywhere
FP32_CFG = dict(N=20, C=12, Cq=20, L=2, m1=3, m2=5)


def test_fp32_mode_forward_and_every_gradient_elementwise(env):
    torch, fno = env
    cfg = fno.FNOConfig(**FP32_CFG)
    y, loss, grads, p, x, t, m = run_gpu_network(torch, fno, cfg, 3, "tc", "f32", 3)
    yo, lo, go = oracle_network(cfg, p, x, t, m)
    err, bound = elementwise_ok(y, yo, 1e-5)
    assert err <= bound, ("y", err, bound)
    assert abs(loss - lo) <= 1e-5 * lo
    for name in ("P", "bp", "W", "b", "R", "Q1", "bq1", "Q2", "bq2"):
        err, bound = elementwise_ok(grads[name], go[name], 1e-5)
        assert err <= bound, (name, err, bound)


# roundings on the longest forward path: the input, then per layer the BF16
# copies of h, S1, U and Wm, then h_L and y1; the backward path adds the BF16
# copies of dy, dz1, dz, dWm, dS2, dS1 and dh per layer
BF16_FWD_ROUNDINGS = lambda L: 1 + 4 * L + 2
BF16_BWD_ROUNDINGS = lambda L: BF16_FWD_ROUNDINGS(L) + 2 + 5 * L


@pytest.mark.parametrize("impl", ["mma", "tc"])
def test_bf16_mode_forward_and_every_gradient_elementwise(env, impl):
    torch, fno = env
    # N 32, C 8, Cq 16: 16-byte aligned operands (staging by whole chunks);
    # 2 m2 = 10: unaligned, element-wise staging
    cfg = fno.FNOConfig(N=32, C=8, Cq=16, L=2, m1=4, m2=5)
    y, loss, grads, p, x, t, m = run_gpu_network(torch, fno, cfg, 2, impl, "bf16", 3)
    yo, lo, go = oracle_network(cfg, p, x, t, m)
    u = 2.0 ** -8
    err, bound = elementwise_ok(y, yo, BF16_FWD_ROUNDINGS(cfg.L) * u)
    assert err <= bound, ("y", err, bound)
    assert abs(loss - lo) <= 2 * BF16_FWD_ROUNDINGS(cfg.L) * u * lo
    for name in ("P", "bp", "W", "b", "R", "Q1", "bq1", "Q2", "bq2"):
        err, bound = elementwise_ok(grads[name], go[name], BF16_BWD_ROUNDINGS(cfg.L) * u)
        assert err <= bound, (name, err, bound)
    if impl == "tc":
        assert tc_flag(fno) == 0


def test_fp32_mode_trains(env):
    torch, fno = env
    cfg = fno.FNOConfig(N=16, C=8, Cq=16, L=2, m1=4, m2=5)
    B = 2
    net = fno.FNO(cfg, batch=B, seed=5, act="f32")
    rng = np.random.default_rng(6)
    rows = B * cfg.N * cfg.N
    xt = torch.tensor(rng.standard_normal((rows, cfg.cin)), dtype=torch.float32, device="cuda")
    tt = torch.tensor(0.1 * rng.standard_normal((rows, cfg.cout)), dtype=torch.float32, device="cuda")
    mt = torch.ones(rows, dtype=torch.float32, device="cuda")
    losses = []
    for _ in range(30):
        net.forward(xt)
        losses.append(float(net.loss(tt, mt)))
        net.backward()
        net.adam(lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]


def test_adam_step_reduces_loss(env):
    torch, fno = env
    cfg = fno.FNOConfig(N=32, C=8, Cq=16, L=2, m1=4, m2=5)
    B = 2
    net = fno.FNO(cfg, batch=B, seed=5)
    rng = np.random.default_rng(6)
    rows = B * cfg.N * cfg.N
    x16 = torch.tensor(rng.standard_normal((rows, cfg.cin)), dtype=torch.bfloat16, device="cuda")
    tt = torch.tensor(0.1 * rng.standard_normal((rows, cfg.cout)), dtype=torch.float32, device="cuda")
    mt = torch.ones(rows, dtype=torch.float32, device="cuda")
    losses = []
    for _ in range(30):
        net.forward(x16)
        losses.append(float(net.loss(tt, mt)))
        net.backward()
        net.adam(lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]


@pytest.mark.parametrize("rows,cols", [(1, 1), (1000, 4), (5000, 32), (777, 128), (300, 300)])
def test_colsum_matches_numpy(env, rows, cols):
    torch, fno = env
    import ctypes
    rng = np.random.default_rng(rows + cols)
    X = rng.standard_normal((rows, cols)).astype(np.float32)
    out0 = rng.standard_normal(cols).astype(np.float32)
    Xt = torch.tensor(X, device="cuda")
    ot = torch.tensor(out0, device="cuda")
    assert fno._lib().rlbm_fno_colsum(ctypes.c_void_p(Xt.data_ptr()), ctypes.c_void_p(ot.data_ptr()),
                                      rows, cols, None) == 0
    torch.cuda.synchronize()
    ref = out0.astype(np.float64) + X.astype(np.float64).sum(0)
    assert np.abs(ot.cpu().numpy() - ref).max() <= 1e-5 * (1 + np.abs(X).sum(0).max())


@pytest.mark.parametrize("impl", ["mma", "tc"])
def test_split_k_weight_gradient_with_ragged_rows(env, impl):
    """out += A^T B over K rows, split into 512-row chunks plus a remainder."""
    torch, fno = env
    net = fno.FNO(fno.FNOConfig(N=8, C=8, Cq=8, L=1, m1=2, m2=2), batch=1, gemm_impl=impl)
    rng = np.random.default_rng(9)
    K, M, N = 1300, 24, 40
    A = bf16_round(rng.standard_normal((K, M)))
    B = bf16_round(rng.standard_normal((K, N)))
    out0 = rng.standard_normal((M, N))
    At = torch.tensor(A, dtype=torch.bfloat16, device="cuda")
    Bt = torch.tensor(B, dtype=torch.bfloat16, device="cuda")
    ot = torch.tensor(out0, dtype=torch.float32, device="cuda")
    net.gemm_tn_sum(At, Bt, M, N, K, ot)
    torch.cuda.synchronize()
    ref = out0 + A.T @ B
    assert np.abs(ot.cpu().numpy() - ref).max() <= 1e-5 * (np.abs(A).T @ np.abs(B)).max() + 1e-5
