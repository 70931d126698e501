"""The serving loop's admission rule, replayed on the host (no GPU): byte budget
never exceeded, arrival order kept, oversize requests dropped."""
import numpy as np
import pytest

from paper_2108_01438_gb300 import mbir


@pytest.fixture(scope="module")
def lib():
    import os
    if not os.path.exists(mbir.LIB_PATH):
        from paper_2108_01438_gb300 import build
        build.build()
    return mbir.lib()


def test_budget_is_never_exceeded_and_order_is_fifo(lib):
    rng = np.random.default_rng(0)
    n = 300
    bytes_ = [int(b) for b in rng.integers(10, 100, n)]
    arrive = sorted(int(a) for a in rng.integers(0, 200, n))
    service = [int(s) for s in rng.integers(1, 30, n)]
    budget = 400
    adm, done, peak = mbir.admission_simulate(budget, bytes_, arrive, service)
    assert peak <= budget
    assert all(a >= t for a, t in zip(adm, arrive))
    assert all(adm[i] <= adm[i + 1] for i in range(n - 1))            # no overtaking
    assert all(d == a + s - 1 for a, d, s in zip(adm, done, service))
    # replay the bytes held per tick independently
    T = max(done) + 1
    held = np.zeros(T, dtype=np.int64)
    for a, d, b in zip(adm, done, bytes_):
        held[a:d + 1] += b
    assert held.max() == peak <= budget


def test_request_larger_than_budget_is_dropped(lib):
    adm, done, peak = mbir.admission_simulate(100, [50, 500, 60], [0, 0, 0], [3, 3, 3])
    assert adm[1] == -1 and done[1] == -1
    assert adm[0] == 0 and adm[2] == 3        # 50 + 60 > 100: the third waits for the first
    assert peak <= 100


def test_everything_fits_means_no_waiting(lib):
    adm, done, peak = mbir.admission_simulate(10 ** 6, [10] * 5, [0, 1, 2, 3, 4], [4] * 5)
    assert adm == [0, 1, 2, 3, 4] and peak == 40
