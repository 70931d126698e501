"""GPU parity of the proximal maps, wavelet transform, step size and FISTA
(through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import fista, isam, wavelet
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RECON_TOL = 1e-3     # reconstruction relative L2 after a fixed number of iterations


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


def _c64(a):
    return torch.from_numpy(np.asarray(a).astype(np.complex64)).cuda()


def _f32(a):
    return torch.from_numpy(np.asarray(a).astype(np.float32)).cuda()


H = wavelet.daubechies_lowpass(4)


@pytest.mark.parametrize("nx,nz", [(64, 256), (32, 64), (48, 96)])
def test_wavelet_transform_matches_oracle(mbir, nx, nz):
    plan = mbir.Plan(W.geometry(nx, nz, 16))
    rng = np.random.default_rng(nx)
    x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    c = plan.wavelet(_c64(x)).cpu().numpy()
    assert _rel(c, wavelet.dwt2(x, H, 3)) <= 1e-6
    xr = plan.wavelet(_c64(c), inverse=True).cpu().numpy()
    assert _rel(xr, x) <= 1e-6
    plan.close()


@pytest.mark.parametrize("penalty", ["l1", "db4"])
def test_prox_matches_oracle(mbir, penalty):
    nx, nz = 64, 256
    plan = mbir.Plan(W.geometry(nx, nz, 16))
    rng = np.random.default_rng(3)
    v = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    v32 = v.astype(np.complex64).astype(np.complex128)
    tau = 0.8
    z = plan.prox(_c64(v), tau, penalty).cpu().numpy()
    ref = fista.prox_l1(v32, tau) if penalty == "l1" else fista.prox_wavelet(v32, tau, H)
    assert _rel(z, ref) <= 1e-6
    # in place
    vt = _c64(v)
    plan.prox(vt, tau, penalty, out=vt)
    assert _rel(vt.cpu().numpy(), ref) <= 1e-6
    plan.close()


@pytest.mark.parametrize("nx,nz", [(32, 32), (40, 72), (96, 160), (136, 64)])
@pytest.mark.parametrize("precision", [0, 2])
def test_db4_prox_small_ragged_and_fp64(mbir, nx, nz, precision):
    """The db4 prox at sizes whose coarse-level tile windows span their block
    several times (nx = 32: an 8-row level-3 block), with ragged tiles
    (136 x 64, 40 x 72), and on FP64 plans."""
    plan = mbir.Plan(W.geometry(nx, nz, 16), precision=precision)
    rng = np.random.default_rng(nx * 7 + nz)
    v = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    tau = 0.7
    if precision == 2:
        vt = torch.from_numpy(v).cuda()
        z = plan.prox(vt, tau, "db4").cpu().numpy()
        assert _rel(z, fista.prox_wavelet(v, tau, H)) <= 1e-11
    else:
        v32 = v.astype(np.complex64).astype(np.complex128)
        z = plan.prox(_c64(v), tau, "db4").cpu().numpy()
        assert _rel(z, fista.prox_wavelet(v32, tau, H)) <= 1e-6
    plan.close()


def _tiny_problem(penalty="l1"):
    wl = W.tiny_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(g.nx, g.m, 0.5, 77)
    clean = isam.phi_nufft(wl["x_true"], mask, g)
    sig = np.sqrt(np.mean(clean[mask == 1] ** 2))
    y = clean + sig * 10 ** (-wl["snr_db"] / 20) * wl["noise"] * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    return d, g, mask, y, phi, phi_adj


def test_lipschitz_matches_oracle(mbir):
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    L_ref = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=300)
    plan = mbir.Plan(d)
    L = plan.lipschitz(torch.from_numpy(mask).cuda(), iters=300)
    assert abs(L - L_ref) <= 1e-4 * L_ref
    plan.close()


@pytest.mark.parametrize("penalty", ["l1", "db4"])
def test_fista_matches_oracle(mbir, penalty):
    """Same lambda and delta on both sides: iterates after 10 and 50 iterations and
    the objective trace agree within the reconstruction tolerance."""
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    L = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=100)
    delta = 1.0 / (1.01 * L)
    if penalty == "l1":
        lam = 0.01 * np.max(np.abs(phi_adj(y * mask)))
        prox = fista.prox_l1
        pen = fista.penalty_l1
    else:
        lam = 0.01 * np.max(np.abs(wavelet.dwt2(phi_adj(y * mask), H, 3)))
        prox = lambda v, t: fista.prox_wavelet(v, t, H)
        pen = lambda x: fista.penalty_wavelet(x, H)
    trace = []
    fista.fista(phi, phi_adj, y, mask, prox, lam, delta, 50, (g.nx, g.nz), trace=trace)
    plan = mbir.Plan(d)
    yt, mt = _f32(y), torch.from_numpy(mask).cuda()
    for iters in (10, 50):
        z, info = plan.solve(yt, mt, penalty=penalty, lam=lam, relative=False, iters=iters, step=delta,
                             trace=True)
        assert _rel(z.cpu().numpy(), trace[iters - 1]) <= RECON_TOL, iters
        assert info["iters"] == iters and info["status"] == 0
    # objective trace: entry k-1 is F(z^{k-1})
    F = [fista.objective(phi, y, mask, np.zeros((g.nx, g.nz)), lam, pen)] + \
        [fista.objective(phi, y, mask, z_, lam, pen) for z_ in trace[:49]]
    assert np.max(np.abs(info["trace"] - np.array(F)) / np.array(F)) <= 1e-4
    F50 = fista.objective(phi, y, mask, trace[49], lam, pen)
    assert abs(info["objective"] - F50) <= 1e-4 * F50
    plan.close()


def test_relative_lambda_rule(mbir):
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    plan = mbir.Plan(d)
    yt, mt = _f32(y), torch.from_numpy(mask).cuda()
    for penalty in ("l1", "db4"):
        _, info = plan.solve(yt, mt, penalty=penalty, lam=0.01, relative=True, iters=2, step=1e-3)
        a = phi_adj(y * mask)
        ref = 0.01 * np.max(np.abs(a if penalty == "l1" else wavelet.dwt2(a, H, 3)))
        assert abs(info["lambda_used"] - ref) <= 1e-5 * ref
    plan.close()


def test_default_step_uses_power_iteration(mbir):
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    plan = mbir.Plan(d)
    _, info = plan.solve(_f32(y), torch.from_numpy(mask).cuda(), iters=3, power_iters=100)
    L_ref = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=100)
    assert abs(info["lipschitz"] - L_ref) <= 1e-3 * L_ref
    assert abs(info["step"] - 1 / (1.01 * info["lipschitz"])) <= 1e-12 * info["step"]
    plan.close()


def test_large_lambda_gives_zero(mbir):
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    plan = mbir.Plan(d)
    z, info = plan.solve(_f32(y), torch.from_numpy(mask).cuda(), lam=1.01, relative=True, iters=5,
                         step=1e-3)
    assert not z.cpu().numpy().any()
    plan.close()


def test_rel_tol_stops_early_and_warm_start_is_near_fixed_point(mbir):
    d, g, mask, y, phi, phi_adj = _tiny_problem()
    plan = mbir.Plan(d)
    yt, mt = _f32(y), torch.from_numpy(mask).cuda()
    z, info = plan.solve(yt, mt, iters=400, min_iter=30, rel_tol=1e-4)
    assert info["status"] == 0 and 30 <= info["iters"] < 400
    z_long, info_long = plan.solve(yt, mt, iters=600)
    z_warm, info_warm = plan.solve(yt, mt, iters=5, x0=z_long)
    assert _rel(z_warm.cpu().numpy(), z_long.cpu().numpy()) <= 1e-3
    assert info_warm["objective"] <= info_long["objective"] * (1 + 1e-5)
    plan.close()


def test_full_size_db4_last_step_matches_oracle(mbir):
    """1024 x 2048 B-scan, db4, 100 iterations (the full-size workload): given the
    GPU's z^98 and z^99, one oracle FISTA step reproduces the GPU's z^100."""
    wl = W.full_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    mask = wl["mask"]
    plan = mbir.Plan(d)
    mt = torch.from_numpy(mask).cuda()
    clean = plan.forward(_c64(wl["x_true"]), mt)
    sig = float(torch.sqrt(torch.mean(clean[mt == 1].double() ** 2)))
    y = clean.double().cpu().numpy() + sig * 10 ** (-wl["snr_db"] / 20) * wl["noise"] * mask
    yt = _f32(y)
    y = yt.double().cpu().numpy()
    _, info = plan.solve(yt, mt, penalty="db4", lam=0.01, iters=1)
    delta, lam = info["step"], info["lambda_used"]
    zs = {}
    for k in (98, 99, 100):
        z, inf = plan.solve(yt, mt, penalty="db4", lam=lam, relative=False, iters=k, step=delta)
        zs[k] = z.cpu().numpy().astype(np.complex128)
    mu = fista.fista_momentum(100)
    x = zs[99] + mu[97] * (zs[99] - zs[98])
    grad = isam.phi_adj_nufft(isam.phi_nufft(x, mask, g) - y * mask, mask, g)
    z100 = fista.prox_wavelet(x - delta * grad, lam * delta, H)
    assert _rel(zs[100], z100) <= 1e-4
    plan.close()


_L_CACHE = {}


@pytest.mark.parametrize("penalty,use_mask", [("l1", True), ("db4", True), ("l1", False)])
def test_fista_ragged_geometry_matches_oracle(mbir, penalty, use_mask):
    """An odd spectral length (m = 75: unpaired columns, a ragged last column tile)
    and a depth whose oversampled transform needs radix 5 (K = 80): the fused
    measurement pass of every iteration and the power iteration against the oracle,
    with a Bernoulli mask and without one."""
    nx, nz, m = 48, 40, 75
    d = W.geometry(nx, nz, m, focus_frac=0.4, disp_edge_rad=15.0)
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(nx, m, 0.6, 91) if use_mask else np.ones((nx, m), dtype=np.uint8)
    x_true = W.point_scatterers(nx, nz, 10, 92)
    clean = isam.phi_nufft(x_true, mask, g)
    y = clean + 0.02 * np.sqrt(np.mean(clean[mask == 1] ** 2)) * W.unit_noise(nx, m, 93) * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    # both power iterations run to convergence (their start vectors differ)
    key = ("ragged", use_mask)
    if key not in _L_CACHE:
        _L_CACHE[key] = fista.power_iteration(phi, phi_adj, (nx, nz), iters=1000)
    L_ref = _L_CACHE[key]
    plan = mbir.Plan(d)
    mt = torch.from_numpy(mask).cuda() if use_mask else None
    L = plan.lipschitz(mt, iters=1000)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    delta = 1.0 / (1.01 * L_ref)
    if penalty == "l1":
        lam = 0.02 * np.max(np.abs(phi_adj(y * mask)))
        prox = fista.prox_l1
    else:
        lam = 0.02 * np.max(np.abs(wavelet.dwt2(phi_adj(y * mask), H, 3)))
        prox = lambda v, t: fista.prox_wavelet(v, t, H)
    trace = []
    fista.fista(phi, phi_adj, y, mask, prox, lam, delta, 30, (nx, nz), trace=trace)
    z, info = plan.solve(_f32(y), mt, penalty=penalty, lam=lam, relative=False, iters=30, step=delta)
    assert info["iters"] == 30 and info["status"] == 0
    assert _rel(z.cpu().numpy(), trace[-1]) <= RECON_TOL
    plan.close()
