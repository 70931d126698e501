"""Pins of the 3-D volume oracle (oracle/volume.py) against facts that do not come
from it: the B-scan oracle it must reduce to, the transpose of its dense matrix,
the isotropy of |q|, and the lateral shift invariance of the model."""
import numpy as np

from oracle import isam, volume
from paper_2108_01438_gb300 import workloads as W


def _vol(nx, ny, nz, m, **kw):
    return volume.make_vol_geom(W.geometry(nx, nz, m, **kw), ny)


def _cx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_a_volume_one_pixel_deep_in_y_is_a_b_scan():
    v = _vol(8, 1, 16, 24)
    rng = np.random.default_rng(1)
    x = _cx(rng, (8, 1, 16))
    y = volume.phi3_exact(x, None, v)
    assert np.max(np.abs(y[:, 0] - isam.phi_exact(x[:, 0], None, v.g))) <= 1e-12 * np.max(np.abs(y))
    r = rng.standard_normal((8, 1, 24))
    a = volume.phi3_adj_exact(r, None, v)
    assert np.max(np.abs(a[:, 0] - isam.phi_adj_exact(r[:, 0], None, v.g))) <= 1e-12 * np.max(np.abs(a))


def test_laterally_constant_in_y_reduces_to_the_b_scan():
    """An image constant along y only excites q_y = 0: every y-row is the B-scan
    response (the 2-D transform of the volume factorises)."""
    v = _vol(8, 6, 16, 24)
    rng = np.random.default_rng(2)
    col = _cx(rng, (8, 16))
    x = np.repeat(col[:, None, :], 6, axis=1)
    y = volume.phi3_exact(x, None, v)
    want = isam.phi_exact(col, None, v.g)
    for py in range(6):
        assert np.max(np.abs(y[:, py] - want)) <= 1e-11 * np.max(np.abs(want))


def test_adjoint_is_the_dense_transpose():
    v = _vol(4, 3, 8, 6)
    rng = np.random.default_rng(3)
    mask = (rng.random((4, 3, 6)) < 0.7).astype(np.uint8)
    n_in, n_out = 4 * 3 * 8, 4 * 3 * 6
    A = np.zeros((n_out, 2 * n_in))
    for i in range(n_in):
        for part, c in ((0, 1.0), (1, 1j)):
            e = np.zeros(n_in, complex)
            e[i] = c
            A[:, part * n_in + i] = volume.phi3_exact(e.reshape(4, 3, 8), mask, v).ravel()
    r = rng.standard_normal((4, 3, 6))
    a = volume.phi3_adj_exact(r, mask, v).ravel()
    want = A.T @ r.ravel()
    got = np.concatenate([a.real, a.imag])
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def test_swapping_the_lateral_axes_swaps_the_measurements():
    """|q| is isotropic: on a square grid (nx = ny, dx = dy) transposing the image's
    lateral axes transposes the measurements."""
    v = _vol(6, 6, 16, 20)
    rng = np.random.default_rng(4)
    x = _cx(rng, (6, 6, 16))
    y = volume.phi3_exact(x, None, v)
    yt = volume.phi3_exact(np.transpose(x, (1, 0, 2)), None, v)
    assert np.max(np.abs(yt - np.transpose(y, (1, 0, 2)))) <= 1e-11 * np.max(np.abs(y))


def test_lateral_shift_invariance():
    """A circular lateral shift of the image shifts the measurements the same way
    (the model is a lateral convolution)."""
    v = _vol(8, 5, 12, 16)
    rng = np.random.default_rng(5)
    x = _cx(rng, (8, 5, 12))
    y = volume.phi3_exact(x, None, v)
    ys = volume.phi3_exact(np.roll(x, (3, -2), axis=(0, 1)), None, v)
    assert np.max(np.abs(ys - np.roll(y, (3, -2), axis=(0, 1)))) <= 1e-11 * np.max(np.abs(y))


def test_in_focus_point_is_its_interferogram_at_its_a_scan():
    """Without the beam filter and dispersion, a point scatterer in the focal plane
    (beta (z - z_f) = 0 at every |q|) comes back at its own A-scan only, as
    A(k) w(z_f) Re{a e^{-j 2 k z_f}}."""
    nx, ny, nz, m = 6, 5, 16, 24
    d = W.geometry(nx, nz, m, na=0.0, disp_edge_rad=0.0)
    d["z_focus_um"] = 7 * d["dz_um"]
    v = volume.make_vol_geom(d, ny)
    a = 0.8 - 0.6j
    x = np.zeros((nx, ny, nz), complex)
    x[2, 3, 7] = a
    y = volume.phi3_exact(x, None, v)
    g = v.g
    want = g.source * isam.depth_weight(g)[7] * np.real(a * np.exp(-2j * g.k * g.z_f))
    assert np.max(np.abs(y[2, 3] - want)) <= 1e-12 * np.max(np.abs(want))
    y[2, 3] = 0
    assert np.max(np.abs(y)) <= 1e-12 * np.max(np.abs(want))


# ------------------------------------------------ the NUFFT realisation of the volume


def test_nufft_volume_with_ny_one_is_the_b_scan_nufft():
    v = _vol(12, 1, 32, 40)
    rng = np.random.default_rng(11)
    x = _cx(rng, (12, 1, 32))
    mask = (rng.random((12, 1, 40)) < 0.6).astype(np.uint8)
    y = volume.phi3_nufft(x, mask, v)
    want = isam.phi_nufft(x[:, 0], mask[:, 0], v.g)
    assert np.max(np.abs(y[:, 0] - want)) <= 1e-12 * np.max(np.abs(want))
    r = rng.standard_normal((12, 1, 40))
    a = volume.phi3_adj_nufft(r, mask, v)
    want = isam.phi_adj_nufft(r[:, 0], mask[:, 0], v.g)
    assert np.max(np.abs(a[:, 0] - want)) <= 1e-12 * np.max(np.abs(want))


def test_nufft_volume_is_close_to_the_direct_sum():
    """The Kaiser-Bessel NUFFT (J = 6, sigma = 2) against the exact depth sum on a
    volume with both lateral axes excited: the same ~1e-6 gap as the B-scan."""
    v = _vol(6, 5, 32, 40, focus_frac=0.3, disp_edge_rad=12.0)
    rng = np.random.default_rng(12)
    x = _cx(rng, (6, 5, 32))
    mask = (rng.random((6, 5, 40)) < 0.7).astype(np.uint8)
    y, ye = volume.phi3_nufft(x, mask, v), volume.phi3_exact(x, mask, v)
    assert np.linalg.norm(y - ye) / np.linalg.norm(ye) <= 2e-5
    r = rng.standard_normal((6, 5, 40))
    a, ae = volume.phi3_adj_nufft(r, mask, v), volume.phi3_adj_exact(r, mask, v)
    assert np.linalg.norm(a - ae) / np.linalg.norm(ae) <= 2e-5


def test_nufft_volume_adjoint_is_the_dense_transpose():
    v = _vol(4, 3, 8, 6)
    rng = np.random.default_rng(13)
    mask = (rng.random((4, 3, 6)) < 0.7).astype(np.uint8)
    n_in = 4 * 3 * 8
    A = np.zeros((4 * 3 * 6, 2 * n_in))
    for i in range(n_in):
        for part, c in ((0, 1.0), (1, 1j)):
            e = np.zeros(n_in, complex)
            e[i] = c
            A[:, part * n_in + i] = volume.phi3_nufft(e.reshape(4, 3, 8), mask, v).ravel()
    r = rng.standard_normal((4, 3, 6))
    a = volume.phi3_adj_nufft(r, mask, v).ravel()
    want = A.T @ r.ravel()
    assert np.max(np.abs(np.concatenate([a.real, a.imag]) - want)) <= 1e-11 * np.max(np.abs(want))


def test_nufft_volume_axis_swap_and_shift():
    """Isotropy of |q| and lateral shift invariance hold for the NUFFT form too."""
    v = _vol(6, 6, 16, 20)
    rng = np.random.default_rng(14)
    x = _cx(rng, (6, 6, 16))
    y = volume.phi3_nufft(x, None, v)
    yt = volume.phi3_nufft(np.transpose(x, (1, 0, 2)), None, v)
    assert np.max(np.abs(yt - np.transpose(y, (1, 0, 2)))) <= 1e-11 * np.max(np.abs(y))
    ys = volume.phi3_nufft(np.roll(x, (2, -1), axis=(0, 1)), None, v)
    assert np.max(np.abs(ys - np.roll(y, (2, -1), axis=(0, 1)))) <= 1e-11 * np.max(np.abs(y))
