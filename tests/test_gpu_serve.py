"""GPU serving loop: requests admitted by budget and advanced together give the
same result as solved alone, meet their stopping rules and never exceed the budget."""
import numpy as np
import pytest

from oracle import isam
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


REQS = [  # (nx, nz, penalty, iters)
    (64, 256, "l1", 20), (48, 128, "db4", 35), (96, 64, "l1", 12), (64, 256, "db4", 25),
    (32, 96, "l1", 30), (48, 128, "l1", 18),
]


@pytest.fixture(scope="module")
def setup(mbir):
    plans, data = {}, []
    for i, (nx, nz, pen, it) in enumerate(REQS):
        if (nx, nz) not in plans:
            plans[(nx, nz)] = mbir.Plan(W.geometry(nx, nz, nz, focus_frac=0.4))
        g = isam.make_geom(W.geometry(nx, nz, nz, focus_frac=0.4))
        x = W.point_scatterers(nx, nz, 6, 700 + i)
        mask = W.mask_bernoulli(nx, nz, 0.6, 800 + i)
        y = isam.phi_nufft(x, mask, g) + 0.01 * W.unit_noise(nx, nz, 900 + i) * mask
        data.append((plans[(nx, nz)], torch.from_numpy(y.astype(np.float32)).cuda(),
                     torch.from_numpy(mask).cuda(), pen, it))
    yield plans, data
    for p in plans.values():
        p.close()


def _solo(mbir, plan, y, m, pen, it, stream):
    with torch.cuda.stream(stream):
        xs, infos = mbir.solve_batch([plan], [y], [m], penalties=pen, lams=0.02, iters=it, stream=stream)
    stream.synchronize()
    return xs[0].cpu().numpy(), infos[0]


def _serve(mbir, data, budget, stream, stagger=True):
    srv = mbir.Server(budget, stream=stream)
    tickets = {}
    results = {}
    pending = list(range(len(data)))
    steps = 0
    with torch.cuda.stream(stream):
        while len(results) < len(data):
            # requests arrive over the first ticks while others are running
            if pending and (not stagger or steps % 3 == 0):
                i = pending.pop(0)
                plan, y, m, pen, it = data[i]
                tickets[i] = srv.submit(plan, y, m, penalty=pen, lam=0.02, iters=it)
            srv.step()
            steps += 1
            st = srv.stats()
            assert st["bytes_in_use"] <= budget
            for i, t in list(tickets.items()):
                r = srv.poll(t)
                if r is not None:
                    results[i] = (r[0].cpu().numpy(), r[1], r[2])
                    del tickets[i]
            assert steps < 10000
    peak = srv.stats()["peak_bytes"]
    srv.close()
    return results, peak


def test_served_results_equal_solo_solves(mbir, setup):
    plans, data = setup
    stream = torch.cuda.Stream()
    results, peak = _serve(mbir, data, 1 << 40, stream)
    for i, (plan, y, m, pen, it) in enumerate(data):
        solo, info = _solo(mbir, plan, y, m, pen, it, stream)
        served, sinfo, lat = results[i]
        assert sinfo["iters"] == it and sinfo["status"] == 0
        assert sinfo["step"] == info["step"] and sinfo["lambda_used"] == info["lambda_used"]
        assert np.array_equal(served, solo), i
        assert lat > 0


def test_small_budget_serialises_but_stays_correct(mbir, setup):
    plans, data = setup
    stream = torch.cuda.Stream()
    per = [mbir.request_bytes(p, pen, it) for p, _, _, pen, it in data]
    budget = max(per) + min(per)          # at most two requests at a time
    results, peak = _serve(mbir, data, budget, stream, stagger=False)
    assert peak <= budget
    for i, (plan, y, m, pen, it) in enumerate(data):
        solo, _ = _solo(mbir, plan, y, m, pen, it, stream)
        assert np.array_equal(results[i][0], solo), i


def test_relative_tolerance_stops_early(mbir, setup):
    plans, data = setup
    stream = torch.cuda.Stream()
    plan, y, m, pen, _ = data[0]
    srv = mbir.Server(1 << 40, stream=stream)
    with torch.cuda.stream(stream):
        t = srv.submit(plan, y, m, penalty="l1", lam=0.02, iters=500, min_iter=10, rel_tol=1e-4)
        r = None
        for _ in range(600):
            srv.step()
            r = srv.poll(t)
            if r is not None:
                break
    srv.close()
    assert r is not None
    assert r[1]["status"] == 0 and 10 <= r[1]["iters"] < 500
    assert np.isfinite(r[1]["objective"]) and r[1]["objective"] > 0


def test_request_larger_than_budget_fails(mbir, setup):
    plans, data = setup
    stream = torch.cuda.Stream()
    plan, y, m, pen, it = data[0]
    srv = mbir.Server(1024, stream=stream)
    with torch.cuda.stream(stream):
        t = srv.submit(plan, y, m, penalty=pen, iters=it)
        srv.step()
        r = srv.poll(t)
    srv.close()
    assert r is not None and r[1]["status"] == -3
