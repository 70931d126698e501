"""Pins of the oracle's orthonormal Daubechies wavelet against its defining
properties (the paper's wavelet-sparsity penalty, Sec. 2.2)."""
import numpy as np
import pytest

from oracle import wavelet


def test_db4_filter_identities():
    h = wavelet.daubechies_lowpass(4)
    assert len(h) == 8
    assert abs(h.sum() - np.sqrt(2)) < 1e-14
    # orthonormal to its own even shifts
    for s in range(4):
        assert abs(np.dot(h[: 8 - 2 * s], h[2 * s:]) - (1.0 if s == 0 else 0.0)) < 1e-13
    # exactly four vanishing moments of the high-pass
    g = wavelet.quadrature_mirror(h)
    n = np.arange(8)
    for p in range(4):
        assert abs(np.sum(n ** p * g)) < 1e-11
    assert abs(np.sum(n ** 4 * g)) > 1.0
    # four zeros at z = -1 and the remaining ones strictly inside the unit circle
    # (minimum phase); the multiple root is split off by exact division
    quot, rem = np.polydiv(h, np.poly(-np.ones(4)))
    assert np.max(np.abs(rem)) < 1e-13
    assert np.all(np.abs(np.roots(quot)) < 1.0)


def test_two_moment_filter_is_the_closed_form_d4():
    """With two vanishing moments the construction gives Daubechies' closed form
    (1+sqrt3, 3+sqrt3, 3-sqrt3, 1-sqrt3) / (4 sqrt2)."""
    r3 = np.sqrt(3.0)
    expect = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * np.sqrt(2.0))
    assert np.max(np.abs(wavelet.daubechies_lowpass(2) - expect)) < 1e-14


def test_one_moment_filter_is_haar():
    assert np.max(np.abs(wavelet.daubechies_lowpass(1) - np.array([1, 1]) / np.sqrt(2))) < 1e-15


@pytest.mark.parametrize("shape", [(64, 256), (32, 64)])
def test_dwt2_orthonormal_and_invertible(shape):
    h = wavelet.daubechies_lowpass(4)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    c = wavelet.dwt2(x, h, 3)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
    assert np.linalg.norm(wavelet.idwt2(c, h, 3) - x) <= 1e-13 * np.linalg.norm(x)
    d = rng.standard_normal(shape)
    assert np.linalg.norm(wavelet.dwt2(wavelet.idwt2(d, h, 3), h, 3) - d) <= 1e-13 * np.linalg.norm(d)


def test_haar_constant_image_lands_in_coarsest_band():
    """A constant image under three Haar levels: every coefficient of the coarsest
    low-low band is 2^3 times the constant, every detail is zero."""
    h = wavelet.daubechies_lowpass(1)
    x = np.full((32, 64), 1.5)
    c = wavelet.dwt2(x, h, 3)
    assert np.allclose(c[:4, :8], 1.5 * 8.0, atol=1e-13)
    c[:4, :8] = 0
    assert np.max(np.abs(c)) < 1e-13


def test_mallat_layout_axes():
    """An image varying only in depth (second index) has no lateral detail: the
    bands that are high-pass along p (lower half of the array) vanish at level 1."""
    h = wavelet.daubechies_lowpass(4)
    x = np.tile(np.random.default_rng(0).standard_normal(64), (32, 1))
    c = wavelet.dwt2(x, h, 1)
    assert np.max(np.abs(c[16:, :])) < 1e-13
    assert np.max(np.abs(c[:16, 32:])) > 1e-3
