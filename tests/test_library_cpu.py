"""Host-side checks of the C ABI library (no GPU needed).

* the library builds and loads, and exports every function declared in
  include/rlbm.h;
* the host-only quadrature refinement agrees with the oracle's (stored in
  tests/golden/quadrature_refined.txt by tests/golden/make_golden.py);
* argument validation (rlbm_workspace_size touches no device);
* the massive-particle quadrature (host-only solve, Sec. 2.3) equals the
  oracle's: the same v0, interval and weights.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1804_02418_gb300 import fno, massive, rlbm, workloads  # fno, massive register their exports

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_02418_gb300 import build
    build.build()
    return rlbm.load_library()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(rlbm_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in rlbm.EXPORTS, f"{n} has no binding"


def test_library_quadrature_matches_oracle_golden(lib):
    w1, w2, p0 = rlbm.quadrature()
    g = np.loadtxt(os.path.join(ROOT, "tests", "golden", "quadrature_refined.txt"), comments="#")
    assert np.allclose(w1, g[:, 1], rtol=1e-14, atol=0)
    assert np.allclose(w2, g[:, 2], rtol=1e-14, atol=0)
    # minimum-norm refinement in absolute units: the smallest shell energy
    # (1.6e-5) is fixed to ~1e-16 absolute by either side's rounding
    assert np.allclose(p0, g[:, 3], rtol=1e-14, atol=1e-15)


def _cfg(samples, prec=1):
    arr = (rlbm._Sample * len(samples))(*[rlbm._to_c_sample(s) for s in samples])
    cfg = rlbm._Config()
    cfg.prec = prec
    cfg.nsamples = len(samples)
    cfg.samples = arr
    return cfg, arr


def _size(lib, samples, prec=1):
    cfg, keep = _cfg(samples, prec)
    n = ctypes.c_size_t()
    rc = lib.rlbm_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
    return rc, n.value


def test_workspace_size_counts_two_population_buffers(lib):
    s = workloads.graphene_sample()
    for prec, es in ((0, 8), (1, 4), (2, 2), (3, 2)):
        rc, n = _size(lib, [s], prec)
        assert rc == 0
        pops = 2 * 48 * s.nx * s.ny * es
        assert pops <= n <= pops * 1.05 + 60 * s.nx * s.ny


@pytest.mark.parametrize("bad", [
    dict(nx=10), dict(ny=5), dict(tau=0.5), dict(tau=0.2), dict(Fx=0.02),
])
def test_invalid_samples_are_rejected(lib, bad):
    s = workloads.graphene_sample(nx=64, ny=32, contact_spacing=24, contact_width=8)
    for k, v in bad.items():
        setattr(s, k, v)
    rc, _ = _size(lib, [s])
    assert rc == -1
    assert lib.rlbm_last_error(None)


def test_invalid_contacts_are_rejected(lib):
    C = workloads.Contact
    cases = [
        workloads.Sample(32, 32, contacts=[C(0, 30, 5)]),                 # off the edge
        workloads.Sample(32, 32, periodic_y=True, contacts=[C(0, 3, 5)]), # periodic edge
        workloads.Sample(32, 32, contacts=[C(4, 3, 5)]),                  # no such edge
        workloads.Sample(32, 32, contacts=[C(0, 3, 0)]),                  # empty
    ]
    for s in cases:
        rc, _ = _size(lib, [s])
        assert rc == -1


def test_bad_precision_and_empty_config(lib):
    s = workloads.shear_wave(16)
    rc, _ = _size(lib, [s], prec=7)
    assert rc == -1
    cfg = rlbm._Config()
    cfg.prec = 1
    cfg.nsamples = 0
    n = ctypes.c_size_t()
    assert lib.rlbm_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == -1


def test_massive_quadrature_matches_the_oracle(lib):
    from oracle import massive as M
    q = M.quadrature()
    got = massive.quadrature()
    assert got["v0"] == q["v0"]
    assert np.allclose(got["window"], q["window"], rtol=1e-15, atol=0)
    assert np.allclose(got["w"], q["w_class"], rtol=1e-13, atol=0)
    assert np.allclose(got["p0"], q["p0_class"], rtol=1e-15, atol=0)
    assert np.array_equal(massive.stencil(), q["n"])


@pytest.mark.parametrize("bad", [dict(nx=4), dict(ny=200000), dict(tau=0.5), dict(Fx=0.02),
                                 dict(prec=2)])
def test_massive_invalid_configs_are_rejected(lib, bad):
    cfg = massive._Config()
    cfg.nx, cfg.ny, cfg.tau, cfg.prec = 32, 16, 1.0, 1
    for k, v in bad.items():
        setattr(cfg, k, v)
    ctx = ctypes.c_void_p()
    assert lib.rlbm_massive_create(ctypes.byref(cfg), ctypes.byref(ctx)) == -1
    assert not ctx.value
    assert lib.rlbm_massive_last_error(None)


def test_residual_decay_fit_recovers_a_known_rate():
    """warmstart.decay_rates fits r(t) ~ C exp(-lambda t) per sample."""
    from paper_1804_02418_gb300 import warmstart as ws
    h = [np.array([1e-3, 2e-3]) * np.exp(-0.01 * 25 * k) for k in range(1, 60)]
    assert np.allclose(ws.decay_rates(h, 25), 0.01, rtol=1e-10)


def test_c_abi_from_plain_c(lib, tmp_path):
    """A C program linked against librlbm.so (no Python, no torch) gets the
    same quadratures as the oracle and the same argument checks."""
    import shutil
    import subprocess
    from oracle import massive as M
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_1804_02418_gb300", "lib")
    exe = str(tmp_path / "host_calls")
    r = subprocess.run([cc, os.path.join(ROOT, "tests", "c_abi", "host_calls.c"),
                        "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lrlbm",
                        "-Wl,-rpath," + libdir, "-Wl,--allow-shlib-undefined", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    lines = {l.split()[0]: l.split()[1:] for l in out.stdout.splitlines()}
    w1, w2, p0 = rlbm.quadrature()
    rc, a, b, c = lines["quadrature"]
    assert rc == "0" and float(a) == w1[0] and float(b) == w2[0] and float(c) == p0[1]
    q = M.quadrature()
    rc, v0, lo, hi, w0 = lines["massive_quadrature"]
    assert rc == "0" and float(v0) == q["v0"] and float(w0) == pytest.approx(q["w_class"][0], rel=1e-13)
    assert lines["stencil"] == ["0", "1", "0", "0", "0"]
    assert lines["massive_create_bad"] == ["-1", "1", "msg"]
    assert lines["workspace_bad"] == ["-1", "msg"]
    assert lines["workspace_ok"][0] == "0" and int(lines["workspace_ok"][1]) >= 2 * 48 * 64 * 32 * 4
