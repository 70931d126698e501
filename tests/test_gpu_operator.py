"""GPU parity of Phi and Phi^H (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

from _parity import assert_parity
from oracle import isam
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5          # operator relative L2 against the FP64 NUFFT oracle (FP32 path)


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(nx, nz, m, seed, keep=0.6, **kw):
    d = W.geometry(nx, nz, m, **kw)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    y = rng.standard_normal((nx, m))
    mask = W.mask_bernoulli(nx, m, keep, seed + 1)
    return d, x, y, mask


def _run(mbir, d, x, y, mask, precision=0):
    plan = mbir.Plan(d, precision=precision)
    cdt = torch.complex128 if precision == 2 else torch.complex64
    rdt = torch.float64 if precision == 2 else torch.float32
    xt = torch.from_numpy(x).to(cdt).cuda()
    yt = torch.from_numpy(y).to(rdt).cuda()
    mt = None if mask is None else torch.from_numpy(mask).cuda()
    yg = plan.forward(xt, mt).double().cpu().numpy()
    xg = plan.adjoint(yt, mt).cpu().numpy().astype(np.complex128)
    plan.close()
    return yg, xg


@pytest.mark.parametrize("nx,nz,m", [(64, 256, 256), (16, 64, 48), (32, 128, 200)])
def test_operator_matches_oracle(mbir, nx, nz, m):
    d, x, y, mask = _case(nx, nz, m, 10 + nx)
    g = isam.make_geom(d)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    yg, xg = _run(mbir, d, x, y, mask)
    assert_parity(yg, isam.phi_nufft(x32, mask, g), OP_TOL, what="Phi")
    assert_parity(xg, isam.phi_adj_nufft(y32, mask, g), OP_TOL, what="Phi^H")
    assert np.all(yg[mask == 0] == 0)


@pytest.mark.parametrize("nx,nz,m", [(6, 24, 37), (10, 40, 53), (14, 56, 29), (12, 60, 90), (2, 8, 5)])
def test_odd_radix_and_ragged_sizes(mbir, nx, nz, m):
    """Lateral widths and depths with radix-3/5/7 factors, ragged spectra, the smallest grid."""
    d, x, y, mask = _case(nx, nz, m, 100 + nx)
    g = isam.make_geom(d)
    yg, xg = _run(mbir, d, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    assert_parity(yg, isam.phi_nufft(x32, mask, g), OP_TOL, what=f"Phi {nx}x{nz}x{m}")
    assert_parity(xg, isam.phi_adj_nufft(y32, mask, g), OP_TOL, what=f"Phi^H {nx}x{nz}x{m}")


@pytest.mark.parametrize("nx,nz,m", [(4096, 16, 16), (8, 4096, 4096), (6, 4096, 3000)])
def test_maximum_sizes(mbir, nx, nz, m):
    """The largest sizes a plan takes: 4096 A-scans (a 4096-point lateral transform
    on two-column tiles) and 4096 depth pixels (K = 8192, the largest row transform,
    where the row kernels fall back from the paired gather by footprint), also with
    a spectrometer length that is not the depth."""
    d, x, y, mask = _case(nx, nz, m, 7 + nx + nz)
    g = isam.make_geom(d)
    yg, xg = _run(mbir, d, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    assert_parity(yg, isam.phi_nufft(x32, mask, g), OP_TOL, what=f"Phi {nx}x{nz}x{m}")
    assert_parity(xg, isam.phi_adj_nufft(y32, mask, g), OP_TOL, what=f"Phi^H {nx}x{nz}x{m}")


def test_gpu_adjoint_identity(mbir):
    d, x, y, mask = _case(64, 256, 256, 3)
    yg, xg = _run(mbir, d, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    lhs = float(np.sum(yg * y32))
    rhs = float(np.real(np.vdot(x32, xg)))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_null_mask_equals_all_ones(mbir):
    d, x, y, _ = _case(32, 64, 64, 8)
    ones = np.ones((32, 64), dtype=np.uint8)
    a = _run(mbir, d, x, y, None)
    b = _run(mbir, d, x, y, ones)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_zero_input_gives_zero(mbir):
    d, x, y, mask = _case(16, 32, 24, 9)
    yg, xg = _run(mbir, d, np.zeros_like(x), np.zeros_like(y), mask)
    assert not yg.any() and not xg.any()


def test_fp64_plan_matches_oracle_tightly(mbir):
    d, x, y, mask = _case(32, 64, 80, 12)
    g = isam.make_geom(d)
    yg, xg = _run(mbir, d, x, y, mask, precision=2)
    assert_parity(yg, isam.phi_nufft(x, mask, g), 1e-11, row_tol=1e-9, max_tol=1e-9, what="Phi FP64")
    assert_parity(xg, isam.phi_adj_nufft(y, mask, g), 1e-11, row_tol=1e-9, max_tol=1e-9, what="Phi^H FP64")


def test_nufft_gap_to_exact_ndft_is_stated(mbir):
    """The GPU operator against the exact NDFT: the KB NUFFT gap (about 5e-6 at J=6)
    plus the FP32 error stays under 2e-5."""
    d, x, y, mask = _case(64, 256, 256, 21)
    g = isam.make_geom(d)
    yg, xg = _run(mbir, d, x, y, mask)
    assert _rel(yg, isam.phi_exact(x, mask, g)) <= 2e-5
    assert _rel(xg, isam.phi_adj_exact(y, mask, g)) <= 2e-5


def test_full_size_operator_elementwise(mbir):
    """1024 x 2048 B-scan (the full-size workload) against the FP64 NUFFT oracle,
    every element, plus sampled outputs against the exact direct sum."""
    wl = W.full_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    x = wl["x_true"]
    mask = wl["mask"]
    y = np.random.default_rng(5).standard_normal((g.nx, g.m))
    yg, xg = _run(mbir, d, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    y_ref = isam.phi_nufft(x32, mask, g)
    # global, per lateral-frequency row (rows 0 and nx/2 run unpaired) and max-element bounds
    assert_parity(yg, y_ref, OP_TOL, what="Phi 1024x2048")
    assert_parity(xg, isam.phi_adj_nufft(y32, mask, g), OP_TOL, what="Phi^H 1024x2048")
    rng = np.random.default_rng(6)
    rows = np.nonzero(mask[:, 0])[0]
    ps = rng.choice(rows, 24)
    ms = rng.integers(0, g.m, 24)
    exact = isam.phi_exact_at(x32, g, ps, ms)
    scale = np.sqrt(np.mean(y_ref[mask == 1] ** 2))
    assert np.max(np.abs(yg[ps, ms] - exact)) <= 1e-4 * scale
