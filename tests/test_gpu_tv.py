"""GPU parity of the isotropic TV penalty (Sec. 2.2): its prox (mbir_prox_tv and
mbir_prox with MBIR_PENALTY_TV) and FISTA with it (mbir_solve), through the C ABI,
against the FP64 oracle (oracle/tv.py)."""
import numpy as np
import pytest

from oracle import fista, isam, tv
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROX_TOL = 2e-5        # FP32 prox after 20-100 dual steps, relative L2
RECON_TOL = 1e-3       # FISTA iterates against the oracle


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


def _img(shape, seed):
    rng = np.random.default_rng(seed)
    # piecewise-constant blocks plus noise: TV has work to do on edges and flats
    base = np.kron(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)),
                   np.ones((shape[0] // 4 + 1, shape[1] // 4 + 1)))[: shape[0], : shape[1]]
    return base + 0.2 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


@pytest.mark.parametrize("nx,nz,tau,iters", [(64, 96, 0.3, 20), (35, 50, 0.8, 20), (16, 45, 0.1, 100),
                                             (2, 40, 0.5, 20), (48, 64, 2.0, 50), (35, 50, 0.8, 21),
                                             (20, 70, 0.4, 3), (9, 35, 0.4, 1), (18, 126, 0.6, 2)])
def test_prox_tv_matches_oracle(mbir, nx, nz, tau, iters):
    """Tiles of 8 x 64 (two-step passes) and 16 x 64 (one-step passes) with ragged
    edges in both directions, a two-row image, a
    strong and a weak tau; odd step counts (two-step passes, then one one-step
    pass), a single step, a single two-step pass."""
    plan = mbir.Plan(W.geometry(nx, nz, 16))
    v = _img((nx, nz), 800 + nx)
    v32 = v.astype(np.complex64)
    z = plan.prox_tv(torch.from_numpy(v32).cuda(), tau, iters).cpu().numpy()
    ref = tv.prox_tv(v32.astype(np.complex128), tau, iters)
    assert _rel(z, ref) <= PROX_TOL
    plan.close()


def test_prox_entry_point_and_aliasing(mbir):
    nx, nz, tau = 40, 72, 0.4
    plan = mbir.Plan(W.geometry(nx, nz, 16))
    v = _img((nx, nz), 810).astype(np.complex64)
    ref = tv.prox_tv(v.astype(np.complex128), tau, 20)
    z = plan.prox(torch.from_numpy(v).cuda(), tau, "tv").cpu().numpy()
    assert _rel(z, ref) <= PROX_TOL
    vt = torch.from_numpy(v).cuda()
    plan.prox(vt, tau, "tv", out=vt)            # in place
    assert _rel(vt.cpu().numpy(), ref) <= PROX_TOL
    # tau = 0 and iters = 0 copy the input
    assert np.array_equal(plan.prox_tv(torch.from_numpy(v).cuda(), 0.0, 20).cpu().numpy(), v)
    assert np.array_equal(plan.prox_tv(torch.from_numpy(v).cuda(), tau, 0).cpu().numpy(), v)
    with pytest.raises(mbir.MbirError):
        plan.prox_tv(vt, tau, 20, out=vt)       # the entry point itself wants distinct buffers
    plan.close()


@pytest.mark.parametrize("nx,nz,iters", [(32, 48, 30), (20, 70, 7)])
def test_prox_tv_fp64_plan_is_tight(mbir, nx, nz, iters):
    """FP64 plans (8 x 32 two-step tiles, 16 x 32 one-step tiles), even and odd counts."""
    tau = 0.6
    plan = mbir.Plan(W.geometry(nx, nz, 16), precision=2)
    v = _img((nx, nz), 820)
    z = plan.prox_tv(torch.from_numpy(v).cuda(), tau, iters).cpu().numpy()
    assert _rel(z, tv.prox_tv(v, tau, iters)) <= 1e-11
    plan.close()


@pytest.mark.parametrize("use_mask", [True, False])
def test_fista_tv_matches_oracle(mbir, use_mask):
    """Same lambda, step and inner steps on both sides: iterates after 10 and 30
    iterations and the objective trace F = 1/2 ||Phi z - s y||^2 + lambda TV(z)."""
    nx, nz, m = 48, 64, 80
    d = W.geometry(nx, nz, m, focus_frac=0.45, disp_edge_rad=10.0)
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(nx, m, 0.6, 830) if use_mask else np.ones((nx, m), dtype=np.uint8)
    x_true = np.zeros((nx, nz), complex)
    x_true[10:30, 20:44] = 1.0 + 0.5j
    x_true[30:40, 5:15] = -0.7j
    clean = isam.phi_nufft(x_true, mask, g)
    y = clean + 0.05 * np.sqrt(np.mean(clean[mask == 1] ** 2)) * W.unit_noise(nx, m, 831) * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    L = fista.power_iteration(phi, phi_adj, (nx, nz), iters=300)
    delta = 1.0 / (1.01 * L)
    lam = 0.02 * np.max(np.abs(phi_adj(y * mask)))
    prox = lambda v, t: tv.prox_tv(v, t, 20)
    trace = []
    fista.fista(phi, phi_adj, y, mask, prox, lam, delta, 30, (nx, nz), trace=trace)
    plan = mbir.Plan(d)
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    mt = torch.from_numpy(mask).cuda() if use_mask else None
    for iters in (10, 30):
        z, info = plan.solve(yt, mt, penalty="tv", lam=lam, relative=False, iters=iters, step=delta,
                             trace=True, tv_iters=20)
        assert info["iters"] == iters and info["status"] == 0
        assert _rel(z.cpu().numpy(), trace[iters - 1]) <= RECON_TOL, iters
    F = [fista.objective(phi, y, mask, np.zeros((nx, nz)), lam, tv.tv)] + \
        [fista.objective(phi, y, mask, z_, lam, tv.tv) for z_ in trace[:29]]
    assert np.max(np.abs(info["trace"] - np.array(F)) / np.array(F)) <= 1e-4
    F30 = fista.objective(phi, y, mask, trace[29], lam, tv.tv)
    assert abs(info["objective"] - F30) <= 1e-4 * F30
    # the relative lambda rule for TV is the pixel one, as for l1
    _, info = plan.solve(yt, mt, penalty="tv", lam=0.02, relative=True, iters=1, step=delta)
    assert abs(info["lambda_used"] - lam) <= 1e-5 * lam
    plan.close()
