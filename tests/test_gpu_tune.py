"""GPU tests of the launch-shape autotuner (mbir_plan_autotune / _get_tuning /
_set_tuning, through the C ABI): every choice it can make computes the same
operator as the oracle, the kept choice carries over to later plans of the same
shape class, and a changed tile width resizes the solver's state safely.

The geometries here are used by no other test file, because a recorded tuning
applies to every later plan of its shape class in the process."""
import numpy as np
import pytest

from oracle import fista, isam
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5          # operator relative L2 against the FP64 NUFFT oracle (FP32 path)
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


def _case(nx, nz, m, seed):
    d = W.geometry(nx, nz, m, focus_frac=0.35, disp_edge_rad=12.0)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    y = rng.standard_normal((nx, m))
    mask = W.mask_bernoulli(nx, m, 0.6, seed + 1)
    return d, x, y, mask


def _apply(plan, x, y, mask):
    xt = torch.from_numpy(x).to(torch.complex64).cuda()
    yt = torch.from_numpy(y).to(torch.float32).cuda()
    mt = torch.from_numpy(mask).cuda()
    return (plan.forward(xt, mt).double().cpu().numpy(),
            plan.adjoint(yt, mt).cpu().numpy().astype(np.complex128))


def _check_oracle(yg, xg, x, y, mask, g):
    x32 = x.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.float32).astype(np.float64)
    assert _rel(yg, isam.phi_nufft(x32, mask, g)) <= OP_TOL
    assert _rel(xg, isam.phi_adj_nufft(y32, mask, g)) <= OP_TOL


@pytest.mark.parametrize("nx,nz,m", [(40, 96, 120), (56, 72, 101)])
def test_autotune_keeps_the_operator(mbir, nx, nz, m):
    d, x, y, mask = _case(nx, nz, m, 700 + nx)
    g = isam.make_geom(d)
    plan = mbir.Plan(d)
    before = _apply(plan, x, y, mask)
    t = plan.autotune(reps=2)
    assert t["tried"] >= 2 and t["pair_ms"] > 0
    assert t["tile_c"] in (2, 4, 8, 16) and t["lateral_order"] in (0, 1)
    assert t["adjoint_kernel"] in (-1, 1, 2, 4, 5)
    assert plan.tuning() == {k: t[k] for k in ("tile_c", "lateral_order", "adjoint_kernel")}
    after = _apply(plan, x, y, mask)
    _check_oracle(*after, x, y, mask, g)
    # a different launch choice only reorders the arithmetic
    assert _rel(after[0], before[0]) <= 1e-5 and _rel(after[1], before[1]) <= 1e-5
    # plans of the same shape class start from the recorded choice
    other = mbir.Plan(d)
    assert other.tuning() == plan.tuning()
    other.close()
    plan.close()


@pytest.mark.parametrize("tile_c,order,adj", [(2, 0, 2), (2, 1, 1), (4, 1, 4), (8, 0, -1), (4, 0, 5)])
def test_every_choice_matches_the_oracle(mbir, tile_c, order, adj):
    d, x, y, mask = _case(24, 80, 66, 710)
    g = isam.make_geom(d)
    plan = mbir.Plan(d)
    plan.set_tuning(tile_c, order, adj)
    assert plan.tuning() == {"tile_c": tile_c, "lateral_order": order, "adjoint_kernel": adj}
    _check_oracle(*_apply(plan, x, y, mask), x, y, mask, g)
    plan.close()


def test_set_tuning_rejects_what_does_not_fit(mbir):
    d, _, _, _ = _case(24, 80, 66, 711)
    plan = mbir.Plan(d)
    keep = plan.tuning()
    for bad in ((3, 0, -1), (32, 0, -1), (4, 2, -1), (4, 0, 0), (4, 0, 3)):
        with pytest.raises(mbir.MbirError):
            plan.set_tuning(*bad)
    assert plan.tuning() == keep
    plan.close()


def test_solve_after_a_tile_change_matches_the_oracle(mbir):
    """A tile change drops the plan's solver state, whose partial-sum buffers are
    sized by the lateral grid: FISTA afterwards (twice, smaller tile then larger)
    still agrees with the oracle."""
    nx, nz, m = 40, 64, 64
    d, _, _, mask = _case(nx, nz, m, 720)
    g = isam.make_geom(d)
    x_true = W.point_scatterers(nx, nz, 8, 721)
    y = isam.phi_nufft(x_true, mask, g) + 0.01 * W.unit_noise(nx, m, 722) * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    L = fista.power_iteration(phi, phi_adj, (nx, nz), iters=300)
    delta = 1.0 / (1.01 * L)
    lam = 0.02 * np.max(np.abs(phi_adj(y * mask)))
    trace = []
    fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 20, (nx, nz), trace=trace)
    plan = mbir.Plan(d)
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    mt = torch.from_numpy(mask).cuda()
    for tile_c in (8, 2, 16):
        plan.set_tuning(tile_c, 0, -1)
        z, info = plan.solve(yt, mt, penalty="l1", lam=lam, relative=False, iters=20, step=delta)
        assert info["iters"] == 20
        assert _rel(z.cpu().numpy(), trace[-1]) <= RECON_TOL, tile_c
    plan.close()
