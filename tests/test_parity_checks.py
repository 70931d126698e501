"""The local parity checks of the GPU tests catch what a global relative L2 misses
(mistakes planted on the CPU, in oracle output)."""
import numpy as np
import pytest

from _parity import assert_parity, rel_l2
from oracle import isam
from paper_2108_01438_gb300 import workloads as W


@pytest.fixture(scope="module")
def ref():
    d = W.geometry(256, 64, 128)
    g = isam.make_geom(d)
    rng = np.random.default_rng(1)
    return isam.phi_adj_nufft(rng.standard_normal((256, 128)), None, g)


def test_exact_copy_passes(ref):
    r = assert_parity(ref.copy(), ref, 1e-5)
    assert r["global"] == 0 and r["row_max"] == 0 and r["max_over_rms"] == 0


def test_one_wrong_element_is_caught(ref):
    bad = ref.copy()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    bad[17, 5] += 1e-3 * rms                   # 1e-3 of the RMS at one of 16384 elements
    assert rel_l2(bad, ref) < 1e-5             # invisible to the global bound
    with pytest.raises(AssertionError, match="max"):
        assert_parity(bad, ref, 1e-5, row_tol=1.0)
    with pytest.raises(AssertionError):
        assert_parity(bad, ref, 1e-5)


@pytest.mark.parametrize("row", [0, 128])     # the rows the paired kernels run alone
def test_one_wrong_lateral_row_is_caught(ref, row):
    spec = np.fft.fft(ref, axis=0)
    rms_row = np.sqrt(np.mean(np.linalg.norm(spec, axis=1) ** 2))
    e = np.random.default_rng(row).standard_normal(spec.shape[1]) + 0j
    spec[row] += 1e-4 * rms_row * e / np.linalg.norm(e)   # that lateral frequency off by 1e-4 of a row
    bad = np.fft.ifft(spec, axis=0)
    assert rel_l2(bad, ref) < 1e-5
    with pytest.raises(AssertionError, match="lateral row"):
        assert_parity(bad, ref, 1e-5, max_tol=1.0)


def test_uniform_small_error_passes(ref):
    rng = np.random.default_rng(2)
    noise = rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)
    bad = ref + 2e-6 * np.sqrt(np.mean(np.abs(ref) ** 2)) * noise / np.sqrt(2)
    assert_parity(bad, ref, 1e-5)
