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


def test_batch_runs_wide_scans_alone_and_overlaps_the_rest(mbir, batch_case):
    """A scan whose row kernels alone fill every SM three times (nx/2 + 1 >= 3 SMs)
    takes the single-scan path inside the batch, on a stream of its own, while the
    small scans share batched stages on another: the wide scan's result equals its
    solo solve bit for bit, the small scans' results equal those of the batch
    without it, and every result matches the oracle's iterates."""
    scans, plans, ys, ms, pens, xs, infos = batch_case
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nx = min(w for w in W.smooth_widths(8, 4096) if w // 2 + 1 >= 3 * sms)   # mixed-radix width
    assert nx <= 2048
    d, g, mask, y = _scan(7, nx, 64, 64)
    wide = mbir.Plan(d)
    yw, mw = torch.from_numpy(y).cuda(), torch.from_numpy(mask).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out, inf = mbir.solve_batch([plans[0], wide, plans[1]], [ys[0], yw, ys[1]], [ms[0], mw, ms[1]],
                                    penalties=[pens[0], "l1", pens[1]], lams=0.02, iters=40, stream=stream)
        z, zi = wide.solve(yw, mw, penalty="l1", lam=0.02, relative=True, iters=40, stream=stream)
    stream.synchronize()
    assert np.array_equal(out[1].cpu().numpy(), z.cpu().numpy())
    assert inf[1]["step"] == zi["step"] and inf[1]["lambda_used"] == zi["lambda_used"] and inf[1]["iters"] == 40
    assert np.array_equal(out[0].cpu().numpy(), xs[0]) and np.array_equal(out[2].cpu().numpy(), xs[1])
    y64 = y.astype(np.float64)
    ref = fista.fista(lambda v: isam.phi_nufft(v, mask, g), lambda r: isam.phi_adj_nufft(r, mask, g), y64, mask,
                      fista.prox_l1, inf[1]["lambda_used"], inf[1]["step"], 40, (g.nx, g.nz))
    assert _rel(out[1].cpu().numpy(), ref) <= 1e-3
    wide.close()
