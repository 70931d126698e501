"""Guard regions (compute-sanitizer is not available): every output and input of
the C-ABI calls sits inside a larger buffer whose margins hold a canary value,
and after each call the margins must be untouched.  Odd and ragged sizes, where
an index slip would reach past the end of a row or of the array."""
import numpy as np
import pytest

from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAD = 4096                       # elements of margin on each side (keeps 16-byte alignment)
CANARY = -7.25e30


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


class Guarded:
    """A contiguous view of `shape` inside a buffer with PAD canary elements on each side."""

    def __init__(self, shape, dtype, init=None):
        n = int(np.prod(shape))
        fill = complex(CANARY, CANARY) if dtype.is_complex else CANARY
        if dtype == torch.uint8:
            fill = 0xA5
        self.buf = torch.full((n + 2 * PAD,), fill, dtype=dtype, device="cuda")
        self.ref = self.buf[:PAD].clone()
        self.view = self.buf[PAD:PAD + n].view(shape)
        if init is not None:
            self.view.copy_(torch.as_tensor(init).to(dtype))

    def intact(self) -> bool:
        torch.cuda.synchronize()
        n = self.view.numel()
        return torch.equal(self.buf[:PAD], self.ref) and torch.equal(self.buf[PAD + n:], self.ref)


@pytest.mark.parametrize("nx,nz,m", [(6, 24, 35), (10, 40, 75), (14, 56, 28), (32, 64, 80)])
def test_calls_write_nothing_outside_their_buffers(mbir, nx, nz, m):
    d = W.geometry(nx, nz, m)
    plan = mbir.Plan(d)
    rng = np.random.default_rng(nx + m)
    x = Guarded((nx, nz), torch.complex64, rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz)))
    y = Guarded((nx, m), torch.float32, rng.standard_normal((nx, m)))
    mask = Guarded((nx, m), torch.uint8, W.mask_bernoulli(nx, m, 0.6, 3))
    out_x = Guarded((nx, nz), torch.complex64)
    out_y = Guarded((nx, m), torch.float32)
    inputs = (x, y, mask)

    def check(what):
        for g in inputs + (out_x, out_y):
            assert g.intact(), what

    plan.forward(x.view, mask.view, out=out_y.view)
    check("forward")
    plan.adjoint(y.view, mask.view, out=out_x.view)
    check("adjoint")
    plan.adjoint_hilbert(y.view, mask.view, out=out_x.view)
    check("adjoint_hilbert")
    plan.isam_interpolated(y.view, mask.view, out=out_x.view)
    check("isam_interpolated")
    plan.prox_tv(x.view, 0.3, 5, out=out_x.view)
    check("prox_tv")
    for kw in (dict(penalty="l1"), dict(penalty="tv", tv_iters=3), dict(penalty="l1", backprojection="hilbert")):
        plan.solve(y.view, mask.view, iters=4, out=out_x.view, trace=True, **kw)
        check(f"solve {kw}")
    plan.ncc(x.view, out_x.view)
    check("ncc")
    plan.close()


def test_wavelet_and_db4_solve_stay_inside(mbir):
    nx, nz, m = 32, 64, 48          # the wavelet needs sizes divisible by 8
    plan = mbir.Plan(W.geometry(nx, nz, m))
    rng = np.random.default_rng(9)
    x = Guarded((nx, nz), torch.complex64, rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz)))
    y = Guarded((nx, m), torch.float32, rng.standard_normal((nx, m)))
    out_x = Guarded((nx, nz), torch.complex64)
    plan.wavelet(x.view, out=out_x.view)
    assert x.intact() and out_x.intact()
    plan.wavelet(out_x.view, inverse=True, out=x.view)
    assert x.intact() and out_x.intact()
    plan.solve(y.view, None, penalty="db4", iters=3, out=out_x.view)
    assert y.intact() and out_x.intact()
    plan.close()
