"""Precision modes on the 64 x 256 point-scatterer workload: FP32, FP32 with
compensated KB accumulation and FP64 GPU plans against the FP64 oracle, for the
operator and for the reconstruction after 10 / 50 / 100 iterations."""
import numpy as np
import pytest

from oracle import fista, isam
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = {"fp32": 0, "fp32c": 1, "fp64": 2}


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def problem():
    wl = W.tiny_workload()
    g = isam.make_geom(wl["geom"])
    mask = W.mask_bernoulli(g.nx, g.m, 0.5, 31)
    clean = isam.phi_nufft(wl["x_true"], mask, g)
    sig = np.sqrt(np.mean(clean[mask == 1] ** 2))
    y = clean + sig * 10 ** (-wl["snr_db"] / 20) * wl["noise"] * mask
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    L = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=100)
    delta = 1.0 / (1.01 * L)
    lam = 0.01 * np.max(np.abs(phi_adj(y * mask)))
    trace = []
    fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 100, (g.nx, g.nz), trace=trace)
    return wl, g, mask, y, delta, lam, trace


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _tensors(mode, x, y, mask):
    cdt = torch.complex128 if mode == 2 else torch.complex64
    rdt = torch.float64 if mode == 2 else torch.float32
    return (torch.from_numpy(x).to(cdt).cuda(), torch.from_numpy(y).to(rdt).cuda(),
            torch.from_numpy(mask).cuda())


def test_operator_error_per_precision(mbir, problem):
    wl, g, mask, y, delta, lam, trace = problem
    rng = np.random.default_rng(2)
    x = rng.standard_normal((g.nx, g.nz)) + 1j * rng.standard_normal((g.nx, g.nz))
    err = {}
    for name, mode in MODES.items():
        plan = mbir.Plan(wl["geom"], precision=mode)
        xt, yt, mt = _tensors(mode, x, y, mask)
        xin = x if mode == 2 else x.astype(np.complex64).astype(np.complex128)
        yin = y if mode == 2 else y.astype(np.float32).astype(np.float64)
        f = plan.forward(xt, mt).double().cpu().numpy()
        a = plan.adjoint(yt, mt).cpu().numpy().astype(np.complex128)
        err[name] = (_rel(f, isam.phi_nufft(xin, mask, g)), _rel(a, isam.phi_adj_nufft(yin, mask, g)))
        plan.close()
    print("operator relative L2 (forward, adjoint):", err)
    assert max(err["fp64"]) <= 1e-11
    assert max(err["fp32"]) <= 1e-5 and max(err["fp32c"]) <= 1e-5
    assert err["fp32c"][0] <= 1.05 * err["fp32"][0] and err["fp32c"][1] <= 1.05 * err["fp32"][1]


def test_reconstruction_error_per_precision(mbir, problem):
    wl, g, mask, y, delta, lam, trace = problem
    err = {}
    for name, mode in MODES.items():
        plan = mbir.Plan(wl["geom"], precision=mode)
        _, yt, mt = _tensors(mode, np.zeros((1, 1)), y, mask)
        err[name] = []
        for k in (10, 50, 100):
            z, _ = plan.solve(yt, mt, penalty="l1", lam=lam, relative=False, iters=k, step=delta)
            err[name].append(_rel(z.cpu().numpy().astype(np.complex128), trace[k - 1]))
        plan.close()
    print("reconstruction relative L2 after 10/50/100 iterations:", err)
    assert max(err["fp64"]) <= 1e-9
    assert max(err["fp32"]) <= 1e-3 and max(err["fp32c"]) <= 1e-3
