"""GPU parity of the evaluation loop of Sec. 3 through the C ABI: the
direct-ISAM baseline on linearly interpolated measurements
(mbir_isam_interpolated), the NCC of Eq. ncc (mbir_ncc) and the golden-section
lambda search (mbir_lambda_search), against the FP64 oracle
(oracle/evaluate.py)."""
import numpy as np
import pytest

from _parity import assert_parity
from oracle import evaluate, fista, isam
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _masks(nx, m, seed):
    rng = np.random.default_rng(seed)
    bern = (rng.random((nx, m)) < 0.5).astype(np.uint8)
    bern[0] = 0                              # an A-scan without samples
    bern[1] = 0
    bern[1, m // 3] = 1                      # one sample, held everywhere
    partial = np.zeros((nx, m), dtype=np.uint8)
    partial[:, m // 4: m // 4 + m // 2] = 1  # the centre half of the band
    equi = np.zeros((nx, m), dtype=np.uint8)
    equi[:, ::2] = 1                         # every other pixel
    return {"random": bern, "partial": partial, "equispaced": equi}


@pytest.mark.parametrize("nx,nz,m", [(16, 64, 48), (9, 40, 75), (32, 128, 256), (6, 24, 30)])
@pytest.mark.parametrize("pattern", ["random", "partial", "equispaced"])
def test_isam_interpolated_matches_oracle(mbir, nx, nz, m, pattern):
    """The paper's three sub-sampling families, odd m and odd nx, empty and
    single-sample A-scans."""
    d = W.geometry(nx, nz, m)
    g = isam.make_geom(d)
    y = np.random.default_rng(nx + m).standard_normal((nx, m))
    mask = _masks(nx, m, 7 + nx)[pattern]
    y32 = y.astype(np.float32).astype(np.float64)
    plan = mbir.Plan(d)
    got = plan.isam_interpolated(torch.from_numpy(y.astype(np.float32)).cuda(),
                                 torch.from_numpy(mask).cuda()).cpu().numpy().astype(np.complex128)
    assert_parity(got, evaluate.isam_interpolated(y32, mask, g), OP_TOL, what=f"interpolated ISAM {pattern}")
    # no mask: the baseline is Phi* itself
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    assert torch.equal(plan.isam_interpolated(yt), plan.adjoint_hilbert(yt))
    plan.close()


def test_isam_interpolated_fp64_and_full_size(mbir):
    d = W.geometry(32, 64, 80)
    g = isam.make_geom(d)
    y = np.random.default_rng(3).standard_normal((32, 80))
    mask = _masks(32, 80, 4)["random"]
    plan = mbir.Plan(d, precision=2)
    got = plan.isam_interpolated(torch.from_numpy(y).cuda(), torch.from_numpy(mask).cuda()).cpu().numpy()
    assert _rel(got, evaluate.isam_interpolated(y, mask, g)) <= 1e-11
    plan.close()
    # the 1024 x 2048 B-scan with the paper's random pattern, every element
    wl = W.full_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(g.nx, g.m, 0.5, 11)
    y = np.random.default_rng(5).standard_normal((g.nx, g.m))
    y32 = y.astype(np.float32).astype(np.float64)
    plan = mbir.Plan(d)
    got = plan.isam_interpolated(torch.from_numpy(y.astype(np.float32)).cuda(),
                                 torch.from_numpy(mask).cuda()).cpu().numpy().astype(np.complex128)
    assert_parity(got, evaluate.isam_interpolated(y32, mask, g), OP_TOL, what="interpolated ISAM 1024x2048")
    plan.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_ncc_matches_oracle(mbir, precision):
    nx, nz = 40, 72
    d = W.geometry(nx, nz, 16)
    rng = np.random.default_rng(21)
    x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    z = x + 0.7 * (rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz)))
    cdt = np.complex128 if precision == 2 else np.complex64
    x, z = x.astype(cdt), z.astype(cdt)
    plan = mbir.Plan(d, precision=precision)
    xt, zt = torch.from_numpy(x).cuda(), torch.from_numpy(z).cuda()
    r = plan.ncc(xt, zt)
    want = evaluate.ncc(x.astype(np.complex128), z.astype(np.complex128))
    assert abs(r - want) <= 1e-12
    assert abs(plan.ncc(xt, xt) - 1.0) <= 1e-12
    # a constant-magnitude image has no correlation to report
    c = torch.full((nx, nz), 1.0 - 1.0j, dtype=xt.dtype, device="cuda")
    assert plan.ncc(c, zt) == 0.0
    plan.close()


def test_lambda_search_matches_oracle(mbir):
    """Golden-section search over log10(relative lambda) in [-3, 0], 7 solves of
    30 FISTA iterations with the oracle's step: the same sequence of lambdas, the
    same NCC at each (the comparisons it decides on differ by at least 5e-3), the
    same best point, and its reconstruction in x."""
    nx, nz, m = 48, 64, 80
    d = W.geometry(nx, nz, m, focus_frac=0.45, disp_edge_rad=10.0)
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(nx, m, 0.5, 901)
    x_true = W.point_scatterers(nx, nz, 30, 902)
    clean = isam.phi_nufft(x_true, mask, g)
    y = clean + 0.1 * np.sqrt(np.mean(clean[mask == 1] ** 2)) * W.unit_noise(nx, m, 903) * mask
    y = y.astype(np.float32).astype(np.float64)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    L = fista.power_iteration(phi, adj, (nx, nz), iters=300)
    delta = 1.0 / (1.01 * L)
    scale = np.max(np.abs(adj(y * mask)))
    recon = {}

    def f(t):
        recon[t] = fista.fista(phi, adj, y, mask, fista.prox_l1, 10 ** t * scale, delta, 30, (nx, nz))
        return evaluate.ncc(recon[t], x_true)

    bt, bf, hist = evaluate.golden_section_max(f, -3.0, 0.0, 7)
    plan = mbir.Plan(d)
    xt = torch.from_numpy(x_true.astype(np.complex64)).cuda()
    x, info = plan.lambda_search(torch.from_numpy(y.astype(np.float32)).cuda(), torch.from_numpy(mask).cuda(), xt,
                                 lo=-3.0, hi=0.0, n_eval=7, penalty="l1", iters=30, step=delta)
    assert info["evaluations"] == 7
    assert np.allclose(info["trace_lambda_rel"], [10 ** t for t, _ in hist], rtol=1e-12, atol=0)
    assert np.max(np.abs(info["trace_ncc"] - np.array([v for _, v in hist]))) <= 1e-4
    assert abs(info["lambda_rel"] - 10 ** bt) <= 1e-12 * 10 ** bt
    assert abs(info["lam"] - 10 ** bt * scale) <= 1e-5 * 10 ** bt * scale
    assert abs(info["ncc"] - bf) <= 1e-4 and info["step"] == delta
    assert _rel(x.cpu().numpy(), recon[bt]) <= 1e-3
    # MBIR beats the interpolated baseline on this phantom (the comparison of Table 1)
    base = plan.isam_interpolated(torch.from_numpy(y.astype(np.float32)).cuda(), torch.from_numpy(mask).cuda())
    assert info["ncc"] > plan.ncc(base, xt) + 0.3
    plan.close()


def test_lambda_search_derives_the_step_once(mbir):
    """With step <= 0 the first solve runs the power iteration and every later one
    reuses its step; invalid brackets are refused on the host."""
    d = W.geometry(16, 32, 32)
    plan = mbir.Plan(d)
    rng = np.random.default_rng(8)
    y = torch.from_numpy(rng.standard_normal((16, 32)).astype(np.float32)).cuda()
    z = torch.from_numpy((rng.standard_normal((16, 32)) + 1j * rng.standard_normal((16, 32))).astype(np.complex64)).cuda()
    _, info = plan.lambda_search(y, None, z, lo=-2.0, hi=0.0, n_eval=4, penalty="l1", iters=5)
    _, ref = plan.solve(y, None, penalty="l1", lam=0.01, iters=1)
    assert abs(info["step"] - ref["step"]) <= 1e-6 * ref["step"]
    with pytest.raises(mbir.MbirError):
        plan.lambda_search(y, None, z, lo=0.0, hi=0.0, n_eval=4)
    with pytest.raises(mbir.MbirError):
        plan.lambda_search(y, None, z, lo=-1.0, hi=0.0, n_eval=1)
    plan.close()
