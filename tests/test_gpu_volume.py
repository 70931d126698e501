"""The ISAM operator of a 3-D volume (Sec. 2.1 over both lateral axes, the
volumetric acquisition of Sec. 3.1) on the GPU: mbir_volume_plan_create with
mbir_forward / mbir_adjoint through the C ABI, against the FP64 volume oracle
(oracle/volume.py: the KB-NUFFT form within 1e-5, the direct depth sum within the
NUFFT gap), with ny = 1-like reductions to the B-scan path."""
import numpy as np
import pytest

from _parity import rel_l2
from oracle import volume
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


def _cx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _vol_case(nx, ny, nz, m, seed, **kw):
    d = W.geometry(nx, nz, m, **kw)
    v = volume.make_vol_geom(d, ny)
    rng = np.random.default_rng(seed)
    x = _cx(rng, (nx, ny, nz))
    y = rng.standard_normal((nx, ny, m))
    mask = (rng.random((nx, ny, m)) < 0.6).astype(np.uint8)
    return d, v, x, y, mask


def _run(mbir, d, ny, x, y, mask, precision=0):
    plan = mbir.VolumePlan(d, ny, precision=precision)
    cdt = torch.complex128 if precision == 2 else torch.complex64
    rdt = torch.float64 if precision == 2 else torch.float32
    mt = None if mask is None else torch.from_numpy(mask).cuda()
    yg = plan.forward(torch.from_numpy(x).to(cdt).cuda(), mt).double().cpu().numpy()
    xg = plan.adjoint(torch.from_numpy(y).to(rdt).cuda(), mt).cpu().numpy().astype(np.complex128)
    plan.close()
    return yg, xg


def _per_slice(got, ref):
    """Largest relative L2 over the (lx, ly) lateral-frequency rows, each judged
    against max(its own norm, a quarter of the RMS row)."""
    d = np.fft.fft2(got - ref, axes=(0, 1))
    r = np.fft.fft2(ref, axes=(0, 1))
    dn = np.linalg.norm(d, axis=2)
    rn = np.linalg.norm(r, axis=2)
    return float(np.max(dn / np.maximum(rn, 0.25 * np.sqrt(np.mean(rn ** 2)))))


@pytest.mark.parametrize("nx,ny,nz,m", [(16, 12, 64, 80), (8, 8, 32, 48), (10, 6, 40, 56), (12, 7, 32, 40),
                                        (11, 13, 24, 30)])
def test_volume_operator_matches_nufft_oracle(mbir, nx, ny, nz, m):
    """7-smooth, odd (ny = 7: unpaired rows) and prime (Bluestein on both axes) widths."""
    d, v, x, y, mask = _vol_case(nx, ny, nz, m, 100 + nx + ny, focus_frac=0.35, disp_edge_rad=15.0)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    yg, xg = _run(mbir, d, ny, x, y, mask)
    ref_y = volume.phi3_nufft(x32, mask, v)
    ref_x = volume.phi3_adj_nufft(y32, mask, v)
    assert rel_l2(yg, ref_y) <= OP_TOL
    assert rel_l2(xg, ref_x) <= OP_TOL
    assert _per_slice(yg, ref_y) <= 5 * OP_TOL and _per_slice(xg, ref_x) <= 5 * OP_TOL
    assert np.all(yg[mask == 0] == 0)


def test_volume_gap_to_the_direct_sum(mbir):
    d, v, x, y, mask = _vol_case(8, 6, 32, 40, 7)
    yg, xg = _run(mbir, d, 6, x, y, mask)
    assert rel_l2(yg, volume.phi3_exact(x, mask, v)) <= 2e-5
    assert rel_l2(xg, volume.phi3_adj_exact(y, mask, v)) <= 2e-5


def test_volume_fp64_plan_matches_oracle_tightly(mbir):
    d, v, x, y, mask = _vol_case(8, 6, 16, 24, 8)
    yg, xg = _run(mbir, d, 6, x, y, mask, precision=2)
    assert rel_l2(yg, volume.phi3_nufft(x, mask, v)) <= 1e-11
    assert rel_l2(xg, volume.phi3_adj_nufft(y, mask, v)) <= 1e-11


def test_volume_adjoint_identity(mbir):
    d, v, x, y, mask = _vol_case(16, 12, 64, 80, 9)
    yg, xg = _run(mbir, d, 12, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    lhs, rhs = float(np.sum(yg * y32)), float(np.real(np.vdot(x32, xg)))
    # rounding of either side scales with |Phi x| |y| (Cauchy-Schwarz), not with the
    # inner product, which random inputs make small by cancellation
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(yg) * np.linalg.norm(y32)


def test_volume_constant_along_y_reproduces_the_b_scan_path(mbir):
    """An image constant along y excites q_y = 0 only: every y row of Phi x is the
    B-scan operator's output (plan of the same geometry), and Phi^H of measurements
    constant along y is the B-scan adjoint in every y row (the 1/(nx ny) of the
    forward 2-D transform and the unnormalised inverse cancel the factor ny)."""
    nx, ny, nz, m = 16, 6, 64, 80
    d = W.geometry(nx, nz, m)
    rng = np.random.default_rng(10)
    col = _cx(rng, (nx, nz)).astype(np.complex64)
    x = np.repeat(col[:, None, :], ny, axis=1)
    yb = rng.standard_normal((nx, m)).astype(np.float32)
    yv = np.repeat(yb[:, None, :], ny, axis=1)
    vol = mbir.VolumePlan(d, ny)
    bsc = mbir.Plan(d)
    y_vol = vol.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_bsc = bsc.forward(torch.from_numpy(col).cuda()).cpu().numpy()
    a_vol = vol.adjoint(torch.from_numpy(yv).cuda()).cpu().numpy()
    a_bsc = bsc.adjoint(torch.from_numpy(yb).cuda()).cpu().numpy()
    for py in range(ny):
        assert rel_l2(y_vol[:, py], y_bsc) <= 1e-5
        assert rel_l2(a_vol[:, py], a_bsc) <= 1e-5
    vol.close()
    bsc.close()


def test_volume_plan_refuses_the_b_scan_calls(mbir):
    d = W.geometry(8, 16, 24)
    vol = mbir.VolumePlan(d, 4)
    y = torch.zeros((8, 24), dtype=torch.float32, device="cuda")
    x = torch.zeros((8, 16), dtype=torch.complex64, device="cuda")
    import ctypes as C
    L = mbir.lib()
    assert L.mbir_adjoint_hilbert(vol.handle, C.c_void_p(y.data_ptr()), None, C.c_void_p(x.data_ptr()), None) == -2
    assert b"volume plan" in L.mbir_last_error()
    ny = C.c_int32()
    assert L.mbir_volume_dims(vol.handle, C.byref(ny)) == 0 and ny.value == 4
    vol.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-3), (2, 1e-8)])
def test_volume_fista_l1_matches_oracle(mbir, precision, tol):
    """FISTA with the l1 penalty on a volume (mbir_solve on a volume plan) against
    the oracle's FISTA driven by the volume KB-NUFFT operator from the GPU's step
    and lambda; the power iteration's L and the relative lambda against the
    oracle's; the reported objective against the oracle's objective of the
    returned volume."""
    from oracle import fista
    nx, ny, nz, m = 12, 8, 32, 40
    d = W.geometry(nx, nz, m)
    v = volume.make_vol_geom(d, ny)
    rng = np.random.default_rng(91)
    x_true = np.zeros((nx, ny, nz), dtype=np.complex128)
    idx = rng.choice(nx * ny * nz, size=12, replace=False)
    x_true.flat[idx] = np.exp(2j * np.pi * rng.random(12))
    mask = (rng.random((nx, ny, m)) < 0.6).astype(np.uint8)
    y = volume.phi3_nufft(x_true, mask, v) + 0.01 * rng.standard_normal((nx, ny, m)) * mask
    rdt = torch.float64 if precision == 2 else torch.float32
    yq = y.astype(np.float64 if precision == 2 else np.float32).astype(np.float64)
    plan = mbir.VolumePlan(d, ny, precision=precision)
    yt = torch.from_numpy(y).to(rdt).cuda()
    mt = torch.from_numpy(mask).cuda()
    z, info = plan.solve(yt, mt, lam=0.02, relative=True, iters=25, power_iters=60)
    z = z.cpu().numpy().astype(np.complex128)
    phi = lambda a: volume.phi3_nufft(a, mask, v)
    phi_adj = lambda r: volume.phi3_adj_nufft(r, mask, v)
    L_ref = fista.power_iteration(phi, phi_adj, (nx, ny, nz), iters=100)
    assert abs(info["lipschitz"] - L_ref) <= 1e-3 * L_ref
    lam_ref = 0.02 * float(np.max(np.abs(phi_adj(yq))))
    assert abs(info["lambda_used"] - lam_ref) <= 1e-5 * lam_ref
    assert info["iters"] == 25 and info["status"] == 0
    ref = fista.fista(phi, phi_adj, yq, mask, fista.prox_l1, info["lambda_used"], info["step"], 25, (nx, ny, nz))
    assert rel_l2(z, ref) <= tol
    f_ref = fista.objective(phi, yq, mask, z, info["lambda_used"], fista.penalty_l1)
    assert abs(info["objective"] - f_ref) <= 1e-4 * f_ref
    # the same step and absolute lambda given explicitly reproduce the solve exactly
    z2, info2 = plan.solve(yt, mt, lam=info["lambda_used"], relative=False, iters=25, step=info["step"])
    assert np.array_equal(z2.cpu().numpy().astype(np.complex128), z)
    assert info2["lipschitz"] == 0
    plan.close()


def test_volume_solve_refuses_other_options(mbir):
    d = W.geometry(8, 16, 24)
    vol = mbir.VolumePlan(d, 4)
    y = torch.zeros((8, 4, 24), dtype=torch.float32, device="cuda")
    x = torch.zeros((8, 4, 16), dtype=torch.complex64, device="cuda")
    import ctypes as C
    L = mbir.lib()
    for pen, rel_tol in ((1, 0.0), (2, 0.0), (0, 1e-4)):
        o = mbir.SolveOpts(pen, 0.01, 1, 5, 0, rel_tol, 5, 0.0, 0, 0, 0)
        assert L.mbir_solve(vol.handle, C.c_void_p(y.data_ptr()), None, C.byref(o), C.c_void_p(x.data_ptr()),
                            None, None) == -1
        assert b"volume plan" in L.mbir_last_error()
    vol.close()
