"""Pins of the oracle's Hilbert-form back-projection (Eq. back_model) and of the
literal zero-pad / DFT form of Eq. for_model, against facts that do not come from
the oracle: scipy's analytic signal, closed forms of the Hilbert transform, the
factor-two identity with the exact transpose on analytic signals, and the direct
depth sum."""
import numpy as np
import pytest
from scipy import signal

from oracle import isam
from paper_2108_01438_gb300 import workloads as W


@pytest.mark.parametrize("M", [16, 15, 2, 1, 75])
def test_conj_analytic_is_scipys_analytic_signal_conjugated(M):
    """A(r) = r - jH(r) is the conjugate of the analytic signal r + jH(r) that
    scipy.signal.hilbert returns (an independent implementation); the mirrored
    side d = -1 is the analytic signal itself."""
    rng = np.random.default_rng(M)
    r = rng.standard_normal((3, M))
    ref = signal.hilbert(r, axis=-1)
    assert np.max(np.abs(isam.conj_analytic(r, 1) - np.conj(ref))) <= 1e-13
    assert np.max(np.abs(isam.conj_analytic(r, -1) - ref)) <= 1e-13


def test_hilbert_closed_forms():
    M = 64
    m = np.arange(M)
    for f0 in (1, 5, 31):
        ph = 2 * np.pi * f0 * m / M + 0.3
        assert np.max(np.abs(isam.hilbert(np.cos(ph)) - np.sin(ph))) <= 1e-13
        assert np.max(np.abs(isam.hilbert(np.sin(ph)) + np.cos(ph))) <= 1e-13
        # A(cos) is the negative-frequency exponential
        assert np.max(np.abs(isam.conj_analytic(np.cos(ph)) - np.exp(-1j * ph))) <= 1e-13
    # DC and the Nyquist alternation have no quadrature part
    assert np.max(np.abs(isam.hilbert(np.full(M, 2.5)))) <= 1e-14
    assert np.max(np.abs(isam.hilbert((-1.0) ** m))) <= 1e-13
    # H(H r) = -r for r without DC and Nyquist content
    rng = np.random.default_rng(7)
    r = rng.standard_normal(M)
    R = np.fft.fft(r)
    R[0] = 0
    R[M // 2] = 0
    r = np.fft.ifft(R).real
    assert np.max(np.abs(isam.hilbert(isam.hilbert(r)) + r)) <= 1e-13


def _natural_grid(nz, ascending, nx=4):
    """m = 2 nz pixels on a uniform wavenumber grid whose step makes 2 k_m dz =
    2 pi (m + m0)/(2 nz): every depth pixel n then sits on DFT bin -n of the
    spectrometer axis, so a profile without a zero-delay term has a strictly
    one-sided spectrum along m and no twin inside the image."""
    M, dz, m0 = 2 * nz, 0.75, 40
    mm = np.arange(M) if ascending else np.arange(M)[::-1]
    k = np.pi * (mm + m0) / (2 * nz * dz)
    return isam.make_geom(dict(nx=nx, nz=nz, m=M, k=k, source=None, dx_um=1.0, dz_um=dz, na=0.1,
                               z_focus_um=3.0, disp_a=0.0, disp_b=0.0, k0=0.0,
                               falloff_half_um=20.0, kb_width=6, kb_oversamp=2.0, kb_alpha=0.0))


def _flat_image(g, seed):
    """Laterally constant image (only q = 0, where beta = 2k) without a zero-delay
    term."""
    rng = np.random.default_rng(seed)
    col = rng.standard_normal(g.nz) + 1j * rng.standard_normal(g.nz)
    col[0] = 0
    return np.tile(col, (g.nx, 1))


@pytest.mark.parametrize("ascending", [True, False])
@pytest.mark.parametrize("which,tol", [("exact", 1e-12), ("nufft", 1e-5)])
def test_back_projection_is_twice_the_transpose_on_analytic_signals(ascending, which, tol):
    """With B x one-sided along m, A(Re{B x}) = B x and B^H conj(B x) = 0, so
    Phi*(Phi x) = B^H B x = 2 Phi^H Phi x: the paper's back-projection is twice
    the exact transpose there, on either wavenumber direction."""
    g = _natural_grid(16, ascending)
    x = _flat_image(g, 3)
    fwd = isam.phi_exact if which == "exact" else isam.phi_nufft
    adj = isam.phi_adj_exact if which == "exact" else isam.phi_adj_nufft
    hil = isam.phi_adj_hilbert_exact if which == "exact" else isam.phi_adj_hilbert_nufft
    y = fwd(x, None, g)
    want = 2 * adj(y, None, g)
    assert np.linalg.norm(hil(y, None, g) - want) <= tol * np.linalg.norm(want)


def test_printed_side_on_a_descending_axis_keeps_only_the_twin():
    """A = Re - jH as printed, applied on a descending wavenumber axis, keeps the
    conjugate of the signal, which B^H maps to zero on the natural grid: the side
    of A has to follow the direction of k."""
    g = _natural_grid(16, ascending=False)
    x = _flat_image(g, 4)
    y = isam.phi_exact(x, None, g)
    printed = isam.b_adj_exact(isam.conj_analytic(y, 1), g)
    assert np.linalg.norm(printed) <= 1e-12 * np.linalg.norm(isam.phi_adj_hilbert_exact(y, None, g))


def test_back_projection_applies_the_mask_before_the_hilbert_transform():
    """Phi*(y) with a mask equals Phi*(s y) without one, and differs from
    applying the mask after A (the transform spreads into unmeasured samples)."""
    g = isam.make_geom(W.geometry(8, 16, 24))
    rng = np.random.default_rng(5)
    y = rng.standard_normal((g.nx, g.m))
    mask = (rng.random((g.nx, g.m)) < 0.5).astype(np.uint8)
    a = isam.phi_adj_hilbert_exact(y, mask, g)
    assert np.max(np.abs(a - isam.phi_adj_hilbert_exact(y * mask, None, g))) <= 1e-12 * np.max(np.abs(a))
    d = 1 if isam.k_increasing(g) else -1
    after = isam.b_adj_exact(mask * isam.conj_analytic(y, d), g)
    assert np.linalg.norm(a - after) > 1e-3 * np.linalg.norm(a)


@pytest.mark.parametrize("shape", [(8, 16, 24), (6, 12, 40), (1, 32, 48)])
def test_literal_pad_and_dft_form_equals_the_direct_depth_sum(shape):
    """Eq. for_model's Q (zero-pad to 2 nz), D (2 nz-point DFT) and K (resampling
    of the padded profile's spectrum onto beta) reproduce the direct depth sum at
    every lateral frequency: the reading that absorbs Q and D loses nothing."""
    nx, nz, m = shape
    g = isam.make_geom(W.geometry(nx, nz, m))
    rng = np.random.default_rng(nx + nz)
    x = rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz))
    want = isam.phi_exact(x, None, g)
    assert np.linalg.norm(isam.phi_qd(x, None, g) - want) <= 1e-11 * np.linalg.norm(want)
