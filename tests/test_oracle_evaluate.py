"""Pins of the evaluation-loop oracle (oracle/evaluate.py): the interpolation,
the NCC of Eq. ncc and the golden-section search, against library routines and
closed forms; the direct ISAM baseline against the physics of an in-focus point."""
import numpy as np
from scipy import interpolate

from oracle import evaluate, isam
from paper_2108_01438_gb300 import workloads as W


def test_interpolation_matches_scipy_and_keeps_measured_samples():
    rng = np.random.default_rng(1)
    y = rng.standard_normal((5, 40))
    mask = (rng.random((5, 40)) < 0.5).astype(np.uint8)
    mask[2] = 0                      # an A-scan without samples stays zero
    mask[3] = 0
    mask[3, 17] = 1                  # a single sample is held everywhere
    out = evaluate.interp_measurements(y, mask)
    assert np.array_equal(out[mask == 1], y[mask == 1])
    assert not out[2].any()
    assert np.all(out[3] == y[3, 17])
    for p in (0, 1, 4):
        idx = np.nonzero(mask[p])[0]
        f = interpolate.interp1d(idx, y[p, idx], kind="linear", bounds_error=False,
                                 fill_value=(y[p, idx[0]], y[p, idx[-1]]))
        assert np.max(np.abs(out[p] - f(np.arange(40)))) <= 1e-12
    # a straight line is reproduced between its first and last measured samples
    line = 0.3 * np.arange(40) - 2.0
    m = np.zeros(40, dtype=np.uint8)
    m[[3, 10, 11, 30]] = 1
    got = evaluate.interp_measurements(line[None, :], m[None, :])[0]
    assert np.max(np.abs(got[3:31] - line[3:31])) <= 1e-12
    assert np.all(got[:3] == line[3]) and np.all(got[31:] == line[30])
    # no mask: unchanged
    assert np.array_equal(evaluate.interp_measurements(y, None), y)


def test_ncc_matches_numpy_corrcoef_and_its_invariances():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 9)) + 1j * rng.standard_normal((6, 9))
    z = rng.standard_normal((6, 9)) + 1j * rng.standard_normal((6, 9))
    want = np.corrcoef(np.abs(x).ravel(), np.abs(z).ravel())[0, 1]
    assert abs(evaluate.ncc(x, z) - want) <= 1e-13
    assert abs(evaluate.ncc(x, x) - 1.0) <= 1e-13
    # magnitudes only: a complex scale and per-pixel phases change nothing
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, x.shape))
    assert abs(evaluate.ncc((2.0 - 1.5j) * x * ph, z) - evaluate.ncc(x, z)) <= 1e-13
    assert abs(evaluate.ncc(x, z) - evaluate.ncc(z, x)) <= 1e-15


def test_golden_section_finds_the_maximum_of_a_unimodal_function():
    t0 = 0.3718
    f = lambda t: -(t - t0) ** 2
    for n in (2, 5, 12, 25):
        t, ft, hist = evaluate.golden_section_max(f, -1.0, 2.0, n)
        assert len(hist) == n
        # the bracket after n evaluations is g^(n-1) of the start; the best point lies in it
        assert abs(t - t0) <= 3.0 * evaluate.INV_PHI ** (n - 1) + 1e-12
        assert ft == max(h[1] for h in hist)
    # the first two points are the golden sections of the interval
    _, _, hist = evaluate.golden_section_max(f, 0.0, 1.0, 2)
    assert abs(hist[0][0] - (1.0 - evaluate.INV_PHI)) <= 1e-15 and abs(hist[1][0] - evaluate.INV_PHI) <= 1e-15
    # each new point reuses one interior point: only one evaluation per step
    calls = []
    evaluate.golden_section_max(lambda t: calls.append(t) or -(t - 0.8) ** 2, 0.0, 1.0, 9)
    assert len(calls) == 9


def test_isam_baseline_focuses_an_in_focus_point():
    """Without dispersion the direct ISAM image of an in-focus point scatterer
    peaks at the scatterer, also from half of the spectrometer samples."""
    nx, nz, m = 32, 64, 64
    d = W.geometry(nx, nz, m, disp_edge_rad=0.0, focus_frac=0.5, falloff=False)
    g = isam.make_geom(d)
    x = np.zeros((nx, nz), complex)
    x[12, 32] = 1.0
    y = isam.phi_exact(x, None, g)
    for mask in (None, W.mask_bernoulli(nx, m, 0.5, 3)):
        r = evaluate.isam_interpolated(y if mask is None else y * mask, mask, g)
        assert np.unravel_index(np.argmax(np.abs(r)), r.shape) == (12, 32)
    # full sampling: the baseline is Phi* itself
    assert np.array_equal(evaluate.isam_interpolated(y, None, g), isam.phi_adj_hilbert_nufft(y, None, g))


def test_isam_baseline_degrades_with_interpolated_samples():
    """The baseline's NCC with a bead phantom is positive and drops when half the
    samples are interpolated instead of measured."""
    nx, nz, m = 32, 64, 64
    g = isam.make_geom(W.geometry(nx, nz, m))
    x = W.point_scatterers(nx, nz, 12, 5)
    r = {}
    for keep in (0.5, 1.0):
        mask = W.mask_bernoulli(nx, m, keep, 6)
        y = isam.phi_exact(x, mask, g)
        r[keep] = evaluate.ncc(evaluate.isam_interpolated(y, mask, g), x)
    assert r[1.0] > r[0.5] > 0.05
