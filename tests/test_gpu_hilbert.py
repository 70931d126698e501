"""GPU parity of the paper's Hilbert-form back-projection Phi*(y) = B^H A(s y)
(Eq. back_model): mbir_adjoint_hilbert and FISTA with it (mbir_solve), through
the C ABI, against the FP64 oracle (oracle/isam.py, oracle/fista.py)."""
import numpy as np
import pytest

from _parity import assert_parity
from oracle import fista, isam, wavelet
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5          # operator relative L2 against the FP64 NUFFT oracle (FP32 path)
RECON_TOL = 1e-3       # FISTA iterates against the oracle
H = wavelet.daubechies_lowpass(4)


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


def _hil(mbir, d, y, mask, precision=0):
    plan = mbir.Plan(d, precision=precision)
    rdt = torch.float64 if precision == 2 else torch.float32
    yt = torch.from_numpy(y).to(rdt).cuda()
    mt = None if mask is None else torch.from_numpy(mask).cuda()
    out = plan.adjoint_hilbert(yt, mt).cpu().numpy().astype(np.complex128)
    plan.close()
    return out


@pytest.mark.parametrize("nx,nz,m", [(64, 256, 256), (16, 64, 48), (6, 24, 35), (10, 40, 75), (14, 56, 28),
                                     (2, 8, 5), (32, 128, 200), (9, 16, 30)])
def test_adjoint_hilbert_matches_oracle(mbir, nx, nz, m):
    """Spectrometer lengths with radix-3/5/7 factors, odd lengths (no Nyquist bin),
    an odd number of A-scans (the last CTA has one); masked."""
    d = W.geometry(nx, nz, m)
    g = isam.make_geom(d)
    rng = np.random.default_rng(nx + m)
    y = rng.standard_normal((nx, m))
    mask = W.mask_bernoulli(nx, m, 0.6, 40 + nx)
    y32 = y.astype(np.float32).astype(np.float64)
    got = _hil(mbir, d, y, mask)
    ref = isam.phi_adj_hilbert_nufft(y32, mask, g)
    assert_parity(got, ref, OP_TOL, what=f"Phi* {nx}x{nz}x{m}")
    # no mask is every sample measured
    assert_parity(_hil(mbir, d, y, None), isam.phi_adj_hilbert_nufft(y32, None, g), OP_TOL, what="Phi* no mask")


def test_unsupported_spectrometer_length_is_refused(mbir):
    d = W.geometry(8, 16, 37)            # 37 is prime: no m-point transform
    plan = mbir.Plan(d)
    y = torch.zeros((8, 37), dtype=torch.float32, device="cuda")
    with pytest.raises(mbir.MbirError) as e:
        plan.adjoint_hilbert(y)
    assert e.value.status == -2
    with pytest.raises(mbir.MbirError) as e:
        plan.solve(y, iters=1, step=0.1, relative=False, backprojection="hilbert")
    assert e.value.status == -2
    # the transpose path is unaffected
    plan.adjoint(y)
    plan.close()


def test_fp64_plan_matches_oracle_tightly(mbir):
    d = W.geometry(32, 64, 80)
    g = isam.make_geom(d)
    rng = np.random.default_rng(12)
    y = rng.standard_normal((32, 80))
    mask = W.mask_bernoulli(32, 80, 0.5, 13)
    assert _rel(_hil(mbir, d, y, mask, precision=2), isam.phi_adj_hilbert_nufft(y, mask, g)) <= 1e-11


@pytest.mark.parametrize("ascending", [True, False])
def test_twice_the_transpose_on_analytic_signals(mbir, ascending):
    """On the natural grid (m = 2 nz uniform wavenumbers) a laterally constant
    image without a zero-delay term gives one-sided A-scans, where
    Phi*(Phi x) = 2 Phi^H Phi x; both sides on the GPU."""
    nz, nx = 16, 4
    M, dz, m0 = 2 * nz, 0.75, 40
    mm = np.arange(M) if ascending else np.arange(M)[::-1]
    d = dict(nx=nx, nz=nz, m=M, k=np.pi * (mm + m0) / (2 * nz * dz), source=None, dx_um=1.0, dz_um=dz,
             na=0.1, z_focus_um=3.0, disp_a=0.0, disp_b=0.0, k0=0.0, falloff_half_um=20.0,
             kb_width=6, kb_oversamp=2.0, kb_alpha=0.0)
    rng = np.random.default_rng(4)
    col = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
    col[0] = 0
    x = torch.from_numpy(np.tile(col, (nx, 1)).astype(np.complex64)).cuda()
    plan = mbir.Plan(d)
    y = plan.forward(x)
    h = plan.adjoint_hilbert(y).cpu().numpy()
    t = plan.adjoint(y).cpu().numpy()
    assert _rel(h, 2 * t) <= 2e-5
    plan.close()


def test_full_size_hilbert_elementwise(mbir):
    """1024 x 2048 B-scan of the full-size workload (half the A-scans measured),
    every element against the FP64 NUFFT oracle."""
    wl = W.full_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    y = np.random.default_rng(5).standard_normal((g.nx, g.m))
    y32 = y.astype(np.float32).astype(np.float64)
    got = _hil(mbir, d, y, wl["mask"])
    assert_parity(got, isam.phi_adj_hilbert_nufft(y32, wl["mask"], g), OP_TOL, what="Phi* 1024x2048")


def _fista_case(use_mask):
    nx, nz, m = 48, 64, 80
    d = W.geometry(nx, nz, m, focus_frac=0.45, disp_edge_rad=10.0)
    g = isam.make_geom(d)
    mask = W.mask_bernoulli(nx, m, 0.6, 830) if use_mask else np.ones((nx, m), dtype=np.uint8)
    x_true = W.point_scatterers(nx, nz, 30, 832)
    clean = isam.phi_nufft(x_true, mask, g)
    y = clean + 0.05 * np.sqrt(np.mean(clean[mask == 1] ** 2)) * W.unit_noise(nx, m, 831) * mask
    return d, g, mask, y.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("penalty", ["l1", "db4"])
@pytest.mark.parametrize("use_mask", [True, False])
def test_fista_with_hilbert_back_projection_matches_oracle(mbir, penalty, use_mask):
    """Same lambda and step on both sides, Phi* in the gradient: iterates after 10
    and 30 iterations and the objective trace."""
    d, g, mask, y = _fista_case(use_mask)
    nx, nz = g.nx, g.nz
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_h = lambda r: isam.phi_adj_hilbert_nufft(r, mask, g)
    L = fista.power_iteration(phi, phi_h, (nx, nz), iters=300)
    delta = 1.0 / (1.01 * L)
    lam = 0.02 * np.max(np.abs(phi_h(y * mask)))
    if penalty == "l1":
        prox, reg = fista.prox_l1, fista.penalty_l1
    else:
        prox = lambda v, t: fista.prox_wavelet(v, t, H)
        reg = lambda z: fista.penalty_wavelet(z, H)
    trace = []
    fista.fista(phi, phi_h, y, mask, prox, lam, delta, 30, (nx, nz), trace=trace)
    plan = mbir.Plan(d)
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    mt = torch.from_numpy(mask).cuda() if use_mask else None
    for iters in (10, 30):
        z, info = plan.solve(yt, mt, penalty=penalty, lam=lam, relative=False, iters=iters, step=delta,
                             trace=True, backprojection="hilbert")
        assert info["iters"] == iters and info["status"] == 0
        assert _rel(z.cpu().numpy(), trace[iters - 1]) <= RECON_TOL, iters
    F = [fista.objective(phi, y, mask, np.zeros((nx, nz)), lam, reg)] + \
        [fista.objective(phi, y, mask, z_, lam, reg) for z_ in trace[:29]]
    assert np.max(np.abs(info["trace"] - np.array(F)) / np.array(F)) <= 1e-4
    plan.close()


def test_step_bound_and_relative_lambda_use_the_hilbert_form(mbir):
    """L from the power iteration on Phi* s Phi and lambda relative to
    max|Phi*(s y)|, each against the oracle."""
    d, g, mask, y = _fista_case(True)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_h = lambda r: isam.phi_adj_hilbert_nufft(r, mask, g)
    L_ref = fista.power_iteration(phi, phi_h, (g.nx, g.nz), iters=600)
    scale = np.max(np.abs(phi_h(y * mask)))
    plan = mbir.Plan(d)
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    mt = torch.from_numpy(mask).cuda()
    _, info = plan.solve(yt, mt, penalty="l1", lam=0.02, relative=True, iters=1, power_iters=300,
                         backprojection="hilbert")
    assert abs(info["lipschitz"] - L_ref) <= 1e-4 * L_ref
    assert abs(info["lambda_used"] - 0.02 * scale) <= 1e-5 * 0.02 * scale
    # the transpose's bound is about half of it on these A-scans
    _, info_t = plan.solve(yt, mt, penalty="l1", lam=0.02, relative=True, iters=1, power_iters=300)
    assert 1.5 < info["lipschitz"] / info_t["lipschitz"] < 2.05
    plan.close()
