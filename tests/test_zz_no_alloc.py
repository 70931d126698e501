"""The allocation-free wavelet entry point (mbir_wavelet_static), for callers that
cannot call cudaMalloc, against the plan-based mbir_wavelet.

Kept in its own file, collected last, so that a stop-at-first-failure run has
already run every other test if this one fails.  It must pass alone in a fresh
process as well as after the other tests (the first call in a context does the
static-scratch set-up); one test runs it in a child process that creates no
plan at all, so the set-up there is the static call's own."""
import ctypes as C
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6   # the tolerance of the wavelet parity tests


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


def _static(mbir, nx, nz, inverse, src, dst):
    stream = torch.cuda.current_stream().cuda_stream
    return mbir.lib().mbir_wavelet_static(nx, nz, int(inverse), C.c_void_p(src.data_ptr()),
                                          C.c_void_p(dst.data_ptr()), C.c_void_p(stream))


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("nx,nz", [(64, 256), (1024, 2048)])
def test_static_wavelet_matches_plan_wavelet_twice(mbir, nx, nz):
    plan = mbir.Plan(W.geometry(nx, nz, 16))
    g = torch.Generator().manual_seed(nx)
    for call in range(2):                      # two calls in a row share the static scratch
        x = torch.complex(torch.randn(nx, nz, generator=g), torch.randn(nx, nz, generator=g)).cuda()
        for inverse in (False, True):
            ref = plan.wavelet(x, inverse=inverse)
            out = torch.empty_like(x)
            assert _static(mbir, nx, nz, inverse, x, out) == 0
            torch.cuda.synchronize()
            assert _rel(out, ref) <= TOL, (call, inverse)
    plan.close()


def test_static_wavelet_rejects_oversize_and_bad_shapes(mbir):
    x = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    assert _static(mbir, 2048, 2048, False, x, y) == -2       # above the 2^21-pixel limit
    assert b"static scratch" in mbir.lib().mbir_last_error()
    assert _static(mbir, 60, 256, False, x, y) == -2          # not divisible by 8
    assert _static(mbir, 64, 256, False, x, x) == -1          # in == out
    torch.cuda.synchronize()


_CHILD = textwrap.dedent("""
    import ctypes as C, sys
    import numpy as np, torch
    sys.path.insert(0, {root!r})
    from oracle import wavelet
    from paper_2108_01438_gb300 import mbir
    lib = mbir.lib()                       # the library only: no plan is ever created
    nx, nz = 64, 96
    h = wavelet.daubechies_lowpass(4)
    rng = np.random.default_rng(7)
    st = torch.cuda.Stream()               # a non-blocking side stream, as torch makes them
    worst = 0.0
    for call in range(2):
        x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
        with torch.cuda.stream(st):
            xt = torch.from_numpy(x.astype(np.complex64)).cuda()
            c = torch.empty_like(xt)
            r = torch.empty_like(xt)
            a = lib.mbir_wavelet_static(nx, nz, 0, C.c_void_p(xt.data_ptr()), C.c_void_p(c.data_ptr()),
                                        C.c_void_p(st.cuda_stream))
            b = lib.mbir_wavelet_static(nx, nz, 1, C.c_void_p(c.data_ptr()), C.c_void_p(r.data_ptr()),
                                        C.c_void_p(st.cuda_stream))
        st.synchronize()
        assert a == 0 and b == 0, (a, b, lib.mbir_last_error())
        x32 = x.astype(np.complex64).astype(np.complex128)
        ref = wavelet.dwt2(x32, h, 3)
        got = c.cpu().numpy().astype(np.complex128)
        worst = max(worst, np.linalg.norm(got - ref) / np.linalg.norm(ref),
                    np.linalg.norm(r.cpu().numpy() - x32) / np.linalg.norm(x32))
    print("WORST", worst)
""")


def test_static_wavelet_first_call_without_any_plan(mbir):
    """A fresh process whose first library call is mbir_wavelet_static, on a
    non-blocking stream: the set-up (address, attributes, taps) is its own, and
    the result matches the FP64 oracle transform on two calls in a row."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=root)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    worst = float(r.stdout.split("WORST")[1].split()[0])
    assert worst <= TOL, worst
