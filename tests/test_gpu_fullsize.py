"""Reconstructions at full size against the FP64 oracle (Eq. alg with the
operator of Eq. for_model):

  - the 1024 x 2048 bead B-scan (half of the A-scans measured, 25 dB, db4,
    3 levels): 100 FISTA iterations with the GPU's own step (power iteration)
    and relative lambda, z^100 against the oracle's z^100 from the same step
    and lambda;
  - B-scans of the uneven-batch sizes (widths up to 2048 A-scans, depths 1024
    and 2048, per-scan focus and dispersion, Bernoulli sub-sampling), solved
    together in one batched launch and each compared with the oracle.

The oracle runs its NUFFT on every host core; these are the slowest GPU tests
(minutes, almost all of it oracle time)."""
import numpy as np
import pytest

from _parity import assert_parity
from oracle import fista, isam, wavelet
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RECON_TOL = 1e-3       # reconstruction relative L2 against the oracle
H = wavelet.daubechies_lowpass(4)


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


def _measure(x_true, mask, g, noise, snr_db):
    """Oracle measurements with noise at snr_db on the measured samples, rounded to FP32."""
    clean = isam.phi_nufft(x_true, mask, g)
    sig = np.sqrt(np.mean(clean[mask == 1] ** 2))
    y = clean + sig * 10 ** (-snr_db / 20) * noise * mask
    return y.astype(np.float32).astype(np.float64)


def test_full_size_db4_reconstruction_matches_oracle(mbir):
    wl = W.full_workload()
    d = wl["geom"]
    g = isam.make_geom(d)
    mask = wl["mask"]
    y = _measure(wl["x_true"], mask, g, wl["noise"], wl["snr_db"])
    plan = mbir.Plan(d)
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    mt = torch.from_numpy(mask).cuda()
    z, info = plan.solve(yt, mt, penalty="db4", lam=0.01, relative=True, iters=100, power_iters=30)
    z = z.cpu().numpy().astype(np.complex128)
    plan.close()
    assert info["iters"] == 100 and info["status"] == 0
    delta, lam = info["step"], info["lambda_used"]
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    lam_ref = 0.01 * np.max(np.abs(wavelet.dwt2(phi_adj(y * mask), H, 3)))
    assert abs(lam - lam_ref) <= 1e-5 * lam_ref
    ref = fista.fista(phi, phi_adj, y, mask, lambda v, t: fista.prox_wavelet(v, t, H), lam, delta, 100,
                      (g.nx, g.nz))
    assert_parity(z, ref, RECON_TOL, what="z^100 1024x2048 db4")
    F = fista.objective(phi, y, mask, ref, lam, lambda x: fista.penalty_wavelet(x, H))
    assert abs(info["objective"] - F) <= 1e-4 * F


# widths and depths of the uneven batch (7-smooth multiples of 8 up to 2048)
BATCH_SHAPES = [(1792, 1024), (2048, 2048), (1280, 1024)]
BATCH_ITERS = 30


def _batch_scan(i, nx, nz):
    rng = np.random.default_rng(W.BASE_SEED + 70 + i)
    d = W.geometry(nx, nz, nz, focus_frac=float(rng.uniform(0.25, 0.75)),
                   disp_edge_rad=float(rng.uniform(-30.0, 30.0)))
    edge = float(np.max(np.abs(d["k"] - d["k0"])))
    d["disp_b"] = float(rng.uniform(-10.0, 10.0)) / edge ** 3
    s = int(rng.integers(1 << 30))
    mask = W.mask_bernoulli(nx, nz, float(rng.uniform(0.25, 0.75)), s + 1)
    g = isam.make_geom(d)
    y = _measure(W.point_scatterers(nx, nz, 200, s), mask, g, W.unit_noise(nx, nz, s + 2), 30.0)
    return d, g, mask, y


def test_batch_scans_of_full_size_match_oracle(mbir):
    scans = [_batch_scan(i, nx, nz) for i, (nx, nz) in enumerate(BATCH_SHAPES)]
    plans = [mbir.Plan(d) for d, _, _, _ in scans]
    ys = [torch.from_numpy(y.astype(np.float32)).cuda() for _, _, _, y in scans]
    ms = [torch.from_numpy(mk).cuda() for _, _, mk, _ in scans]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xs, infos = mbir.solve_batch(plans, ys, ms, penalties="l1", lams=0.01, relative=True,
                                     iters=BATCH_ITERS, power_iters=30, stream=stream)
    stream.synchronize()
    xs = [x.cpu().numpy().astype(np.complex128) for x in xs]
    for p in plans:
        p.close()
    for i, (d, g, mask, y) in enumerate(scans):
        phi = lambda v: isam.phi_nufft(v, mask, g)
        phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
        lam, delta = infos[i]["lambda_used"], infos[i]["step"]
        lam_ref = 0.01 * np.max(np.abs(phi_adj(y * mask)))
        assert abs(lam - lam_ref) <= 1e-5 * lam_ref, i
        ref = fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, BATCH_ITERS, (g.nx, g.nz))
        assert_parity(xs[i], ref, RECON_TOL, what=f"batched scan {i} {g.nx}x{g.nz}")
