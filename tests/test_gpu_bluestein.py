"""Lateral widths that do not factor into radices 2..8 (primes, 2 x prime, ...):
the lateral transform of Eq. 4 runs in the Bluestein (chirp-z) form.  Phi, Phi^H,
the paper's back-projection Phi* and FISTA through the C ABI against the FP64
oracle, whose lateral DFT takes any width."""
import numpy as np
import pytest

from _parity import assert_parity, rel_l2
from oracle import fista, isam
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5          # operator relative L2 against the FP64 NUFFT oracle (FP32 path)
RECON_TOL = 1e-3


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


def _case(nx, nz, m, seed, keep=0.6):
    d = W.geometry(nx, nz, m)
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
    mt = torch.from_numpy(mask).cuda()
    yg = plan.forward(xt, mt).double().cpu().numpy()
    xg = plan.adjoint(yt, mt).cpu().numpy().astype(np.complex128)
    xh = plan.adjoint_hilbert(yt, mt).cpu().numpy().astype(np.complex128)
    plan.close()
    return yg, xg, xh


@pytest.mark.parametrize("nx,nz,m", [(11, 32, 48), (13, 64, 80), (1021, 64, 96), (1031, 32, 40), (22, 40, 64),
                                     (19, 16, 24)])
def test_prime_widths_match_oracle(mbir, nx, nz, m):
    d, x, y, mask = _case(nx, nz, m, 900 + nx)
    g = isam.make_geom(d)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    yg, xg, xh = _run(mbir, d, x, y, mask)
    assert_parity(yg, isam.phi_nufft(x32, mask, g), OP_TOL, what=f"Phi nx={nx}")
    assert_parity(xg, isam.phi_adj_nufft(y32, mask, g), OP_TOL, what=f"Phi^H nx={nx}")
    assert_parity(xh, isam.phi_adj_hilbert_nufft(y32, mask, g), OP_TOL, what=f"Phi* nx={nx}")
    assert np.all(yg[mask == 0] == 0)


def test_prime_width_fp64_plan_matches_oracle_tightly(mbir):
    d, x, y, mask = _case(13, 32, 40, 931)
    g = isam.make_geom(d)
    yg, xg, _ = _run(mbir, d, x, y, mask, precision=2)
    assert rel_l2(yg, isam.phi_nufft(x, mask, g)) <= 1e-11
    assert rel_l2(xg, isam.phi_adj_nufft(y, mask, g)) <= 1e-11


def test_prime_width_adjoint_identity(mbir):
    d, x, y, mask = _case(1021, 32, 48, 941)
    yg, xg, _ = _run(mbir, d, x, y, mask)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    lhs = float(np.sum(yg * y32))
    rhs = float(np.real(np.vdot(x32, xg)))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_fista_at_a_prime_width_matches_oracle(mbir):
    nx, nz, m = 67, 48, 64
    d = W.geometry(nx, nz, m, focus_frac=0.4)
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(nx, m, 0.6, 951)
    x_true = W.point_scatterers(nx, nz, 12, 952)
    clean = isam.phi_nufft(x_true, mask, g)
    y = clean + 0.02 * np.sqrt(np.mean(clean[mask == 1] ** 2)) * W.unit_noise(nx, m, 953) * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    L = fista.power_iteration(phi, phi_adj, (nx, nz), iters=200)
    delta = 1.0 / (1.01 * L)
    lam = 0.02 * np.max(np.abs(phi_adj(y * mask)))
    ref = fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 30, (nx, nz))
    plan = mbir.Plan(d)
    mt = torch.from_numpy(mask).cuda()
    z, info = plan.solve(torch.from_numpy(y.astype(np.float32)).cuda(), mt, penalty="l1", lam=lam,
                         relative=False, iters=30, step=delta)
    assert info["iters"] == 30 and info["status"] == 0
    assert_parity(z.cpu().numpy(), ref, RECON_TOL, what="FISTA nx=67")
    Lg = plan.lipschitz(mt, iters=200)
    assert abs(Lg - L) <= 1e-3 * L
    plan.close()


def test_prime_width_in_a_batch_equals_its_solo_solve(mbir):
    """A Bluestein scan and a mixed-radix scan in one batched launch."""
    shapes = [(37, 64, 80), (48, 64, 80)]
    plans, ys, ms = [], [], []
    for i, (nx, nz, m) in enumerate(shapes):
        d = W.geometry(nx, nz, m)
        g = isam.make_geom(d)
        mask = W.mask_bernoulli(nx, m, 0.5, 960 + i)
        y = isam.phi_nufft(W.point_scatterers(nx, nz, 6, 970 + i), mask, g)
        plans.append(mbir.Plan(d))
        ys.append(torch.from_numpy(y.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xs, infos = mbir.solve_batch(plans, ys, ms, penalties="l1", lams=0.02, iters=20, stream=stream)
    stream.synchronize()
    for i, p in enumerate(plans):
        z, _ = p.solve(ys[i], ms[i], penalty="l1", lam=infos[i]["lambda_used"], relative=False, iters=20,
                       step=infos[i]["step"])
        assert rel_l2(xs[i].cpu().numpy(), z.cpu().numpy()) <= 1e-5, i
    for p in plans:
        p.close()


def test_bluestein_plan_keeps_its_radix_order_and_refuses_too_wide(mbir):
    plan = mbir.Plan(W.geometry(101, 32, 40))
    with pytest.raises(mbir.MbirError):
        plan.set_tuning(2, 1, -1)          # reversed radix order: not for a Bluestein plan
    t = plan.autotune(reps=1)
    assert t["lateral_order"] == 0
    plan.close()
    with pytest.raises(mbir.MbirError) as e:
        mbir.Plan(W.geometry(2053, 16, 16))   # prime above 2048: Bluestein length beyond the tile
    assert e.value.status == -2
