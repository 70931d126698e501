"""The allocation-free wavelet entry point (mbir_wavelet_static), for callers that
cannot call cudaMalloc, against the plan-based mbir_wavelet.

Kept in its own file, collected last, so that a stop-at-first-failure run has
already run every other test if this one fails.  It must pass alone in a fresh
process as well as after the other tests (the first call on a device does the
static-scratch set-up)."""
import ctypes as C

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
