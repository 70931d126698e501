"""GPU batch engine (mbir_solve_batch): uneven B-scans solved together match
their solo solves, the oracle, and do not depend on the batch mix."""
import numpy as np
import pytest

from oracle import fista, isam, wavelet
from paper_2108_01438_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbir():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01438_gb300 import build, mbir as m
    build.build()
    m.lib()
    return m


SHAPES = [(64, 256, 256, "l1"), (48, 128, 160, "db4"), (96, 64, 80, "l1"), (32, 96, 96, "db4")]


def _scan(i, nx, nz, m):
    d = W.geometry(nx, nz, m, focus_frac=0.3 + 0.1 * i, disp_edge_rad=10.0 + 5 * i)
    x = W.point_scatterers(nx, nz, 8, 300 + i)
    mask = W.mask_bernoulli(nx, m, 0.5 + 0.1 * i, 400 + i)
    g = isam.make_geom(d)
    y = isam.phi_nufft(x, mask, g) + 0.01 * W.unit_noise(nx, m, 500 + i) * mask
    return d, g, mask, y.astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def batch_case(mbir):
    scans = [_scan(i, *s[:3]) for i, s in enumerate(SHAPES)]
    plans = [mbir.Plan(d) for d, _, _, _ in scans]
    ys = [torch.from_numpy(y).cuda() for _, _, _, y in scans]
    ms = [torch.from_numpy(mk).cuda() for _, _, mk, _ in scans]
    pens = [s[3] for s in SHAPES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xs, infos = mbir.solve_batch(plans, ys, ms, penalties=pens, lams=0.02, iters=40, stream=stream)
    stream.synchronize()
    yield scans, plans, ys, ms, pens, [x.cpu().numpy() for x in xs], infos
    for p in plans:
        p.close()


def test_batch_matches_solo_solves(mbir, batch_case):
    scans, plans, ys, ms, pens, xs, infos = batch_case
    for i, p in enumerate(plans):
        z, info = p.solve(ys[i], ms[i], penalty=pens[i], lam=infos[i]["lambda_used"], relative=False,
                          iters=40, step=infos[i]["step"])
        assert _rel(xs[i], z.cpu().numpy()) <= 1e-5, i


def test_batch_result_does_not_depend_on_the_mix(mbir, batch_case):
    scans, plans, ys, ms, pens, xs, infos = batch_case
    stream = torch.cuda.Stream()
    for i in (0, 1):
        with torch.cuda.stream(stream):
            alone, inf = mbir.solve_batch([plans[i]], [ys[i]], [ms[i]], penalties=pens[i], lams=0.02, iters=40,
                                          stream=stream)
        stream.synchronize()
        assert np.array_equal(alone[0].cpu().numpy(), xs[i])
        assert inf[0]["step"] == infos[i]["step"] and inf[0]["lambda_used"] == infos[i]["lambda_used"]


def test_batch_matches_oracle(mbir, batch_case):
    scans, plans, ys, ms, pens, xs, infos = batch_case
    H = wavelet.daubechies_lowpass(4)
    for i in (0, 1):
        d, g, mask, y = scans[i]
        y64 = y.astype(np.float64)
        phi = lambda v: isam.phi_nufft(v, mask, g)
        phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
        prox = fista.prox_l1 if pens[i] == "l1" else (lambda v, t: fista.prox_wavelet(v, t, H))
        ref = fista.fista(phi, phi_adj, y64, mask, prox, infos[i]["lambda_used"], infos[i]["step"], 40,
                          (g.nx, g.nz))
        assert _rel(xs[i], ref) <= 1e-3, i


def test_batch_rejects_bad_arguments(mbir, batch_case):
    scans, plans, ys, ms, pens, xs, infos = batch_case
    with pytest.raises(mbir.MbirError):
        mbir.solve_batch([plans[0], plans[0]], [ys[0], ys[0]], iters=5)
