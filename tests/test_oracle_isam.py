"""Pins of the FP64 oracle operators against facts the paper and the mathematics
fix, independently of the oracle's own code paths."""
import numpy as np
import pytest
from scipy import integrate

from oracle import isam
from paper_2108_01438_gb300 import workloads as W


def _geom(nx, nz, m, **kw):
    return isam.make_geom(W.geometry(nx, nz, m, **kw))


def _rand_x(rng, g):
    return rng.standard_normal((g.nx, g.nz)) + 1j * rng.standard_normal((g.nx, g.nz))


def _dense(op, shape_in, complex_in):
    """Real matrix of a real-linear map, column by column."""
    cols = []
    n = int(np.prod(shape_in))
    for part in ((1.0, 1j) if complex_in else (1.0,)):
        for i in range(n):
            e = np.zeros(n, dtype=np.complex128 if complex_in else np.float64)
            e[i] = part
            out = op(e.reshape(shape_in))
            out = np.asarray(out)
            cols.append(np.concatenate([out.real.ravel(), out.imag.ravel()])
                        if np.iscomplexobj(out) else out.ravel())
    return np.array(cols).T


@pytest.mark.parametrize("which", ["exact", "nufft"])
@pytest.mark.parametrize("nx", [4, 11])
def test_adjoint_is_transpose_dense(which, nx):
    """Phi^H must be the transpose of Phi as real matrices (Sec. 2.1, Eq. ls_grad
    needs the true adjoint); also at a prime width (the oracle takes any width, the
    reference for a future arbitrary-width lateral transform)."""
    g = _geom(nx, 8, 8)
    mask = (np.random.default_rng(3).random((nx, 8)) < 0.7).astype(np.uint8)
    fwd = isam.phi_exact if which == "exact" else isam.phi_nufft
    adj = isam.phi_adj_exact if which == "exact" else isam.phi_adj_nufft
    A = _dense(lambda x: fwd(x, mask, g), (g.nx, g.nz), True)      # (M, 2N)
    B = _dense(lambda y: adj(y, mask, g), (g.nx, g.m), False)       # (2N, M)
    assert np.max(np.abs(A.T - B)) <= 1e-13 * np.max(np.abs(A))


@pytest.mark.parametrize("which", ["exact", "nufft"])
def test_adjoint_identity(which):
    """<Phi x, y> = Re <x, Phi^H y> on random seeded inputs, with a mask."""
    g = _geom(64, 256, 256)
    rng = np.random.default_rng(11)
    x = _rand_x(rng, g)
    y = rng.standard_normal((g.nx, g.m))
    mask = W.mask_bernoulli(g.nx, g.m, 0.5, 5)
    fwd = isam.phi_exact if which == "exact" else isam.phi_nufft
    adj = isam.phi_adj_exact if which == "exact" else isam.phi_adj_nufft
    lhs = float(np.sum(fwd(x, mask, g) * y))
    rhs = float(np.real(np.vdot(x, adj(y, mask, g))))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _uniform_k_geometry(nz, m, m0, dz):
    """nx = 1, k_m chosen so that 2 k_m dz = 2 pi (m + m0)/(2 nz); no filter,
    no falloff, focus at zero delay, no dispersion: Phi reduces to the real part of
    a zero-padded 2 nz-point DFT (the Q and D of Eq. for_model)."""
    k = np.pi * (np.arange(m) + m0) / (2 * nz * dz)
    return isam.make_geom(dict(nx=1, nz=nz, m=m, k=k, source=None, dx_um=1.0, dz_um=dz,
                               na=0.0, z_focus_um=0.0, disp_a=0.0, disp_b=0.0, k0=0.0,
                               falloff_half_um=0.0, kb_width=6, kb_oversamp=2.0,
                               kb_alpha=0.0))


@pytest.mark.parametrize("which,tol", [("exact", 1e-12), ("nufft", 2e-5)])
def test_special_case_reduces_to_fft(which, tol):
    nz, m, m0, dz = 32, 48, 40, 0.75
    g = _uniform_k_geometry(nz, m, m0, dz)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, nz)) + 1j * rng.standard_normal((1, nz))
    fwd = isam.phi_exact if which == "exact" else isam.phi_nufft
    adj = isam.phi_adj_exact if which == "exact" else isam.phi_adj_nufft
    spec = np.fft.fft(np.concatenate([x[0], np.zeros(nz)]))
    bins = (np.arange(m) + m0) % (2 * nz)
    expect = spec[bins].real
    got = fwd(x, None, g)[0]
    assert np.linalg.norm(got - expect) <= tol * np.linalg.norm(expect)
    # adjoint: sum_m y_m e^{+j 2 pi (m + m0) n / (2 nz)} for n < nz
    y = rng.standard_normal((1, m))
    acc = np.zeros(2 * nz, dtype=np.complex128)
    np.add.at(acc, bins, y[0])
    expect_adj = (2 * nz * np.fft.ifft(acc))[:nz]
    got_adj = adj(y, None, g)[0]
    assert np.linalg.norm(got_adj - expect_adj) <= tol * np.linalg.norm(expect_adj)


def test_infocus_point_without_beam_filter_is_interferogram():
    """A single reflector at the focal depth with no beam filter (G = 1) yields the
    textbook SD-OCT interferogram A(k) w(z) cos(2 k z_f - Omega(k)) in its own
    A-scan and nothing elsewhere."""
    nx, nz, m = 16, 64, 96
    d = W.geometry(nx, nz, m, na=0.0)
    n_f, p0 = 23, 5
    d["z_focus_um"] = n_f * d["dz_um"]
    g = isam.make_geom(d)
    x = np.zeros((nx, nz), dtype=np.complex128)
    x[p0, n_f] = 1.0
    y = isam.phi_exact(x, None, g)
    k = np.asarray(d["k"])
    omega = d["disp_a"] * (k - d["k0"]) ** 2 + d["disp_b"] * (k - d["k0"]) ** 3
    w = np.exp(-np.log(2) * (d["z_focus_um"] / d["falloff_half_um"]) ** 2)
    expect = np.zeros((nx, m))
    expect[p0] = d["source"] * w * np.cos(2 * k * d["z_focus_um"] - omega)
    assert np.max(np.abs(y - expect)) <= 1e-12
    yn = isam.phi_nufft(x, None, g)
    assert np.linalg.norm(yn - expect) <= 2e-5 * np.linalg.norm(expect)


def test_infocus_point_with_beam_filter_has_depth_independent_blur():
    """At the focal plane the lateral response of every wavenumber is the
    inverse DFT of the beam filter alone: no ISAM (beta) dependence."""
    nx, nz, m = 32, 64, 48
    d = W.geometry(nx, nz, m, na=0.1)
    n_f, p0 = 17, 9
    d["z_focus_um"] = n_f * d["dz_um"]
    g = isam.make_geom(d)
    x = np.zeros((nx, nz), dtype=np.complex128)
    x[p0, n_f] = 1.0
    y = isam.phi_exact(x, None, g)
    k = np.asarray(d["k"])
    lt = np.where(np.arange(nx) < nx / 2, np.arange(nx), np.arange(nx) - nx)
    q = 2 * np.pi * lt / (nx * d["dx_um"])
    omega = d["disp_a"] * (k - d["k0"]) ** 2
    w = np.exp(-np.log(2) * (d["z_focus_um"] / d["falloff_half_um"]) ** 2)
    expect = np.zeros((nx, m))
    for p in range(nx):
        for mm in range(m):
            G = np.exp(-q ** 2 / (2 * k[mm] ** 2 * 0.1 ** 2))
            gm = np.sum(G * np.cos(q * (p - p0) * d["dx_um"])) / nx
            expect[p, mm] = d["source"][mm] * w * gm * np.cos(2 * k[mm] * d["z_focus_um"] - omega[mm])
    assert np.max(np.abs(y - expect)) <= 1e-12


@pytest.mark.parametrize("l0", [3, 13])   # a positive and a negative lateral frequency
def test_plane_wave_follows_isam_dispersion_relation(l0):
    """A single lateral plane wave at one depth: each wavenumber sees the axial
    frequency beta = sqrt(4k^2 - q^2) of Eq. 5 for that wave's q."""
    nx, nz, m = 16, 32, 40
    d = W.geometry(nx, nz, m, na=0.05, focus_frac=0.3)
    g = isam.make_geom(d)
    n1 = 21
    p = np.arange(nx)
    x = np.zeros((nx, nz), dtype=np.complex128)
    x[:, n1] = np.exp(2j * np.pi * l0 * p / nx)
    y = isam.phi_exact(x, None, g)
    lt = l0 if l0 < nx // 2 else l0 - nx
    q = 2 * np.pi * lt / (nx * d["dx_um"])
    k = np.asarray(d["k"])
    beta = np.sqrt(4 * k ** 2 - q ** 2)
    z1, zf = n1 * d["dz_um"], d["z_focus_um"]
    omega = d["disp_a"] * (k - d["k0"]) ** 2
    H = d["source"] * np.exp(-q ** 2 / (2 * k ** 2 * 0.05 ** 2)) * np.exp(1j * omega) * np.exp(-2j * k * zf)
    w = np.exp(-np.log(2) * (z1 / d["falloff_half_um"]) ** 2)
    expect = (np.exp(1j * q * p[:, None] * d["dx_um"]) * H[None, :] * w
              * np.exp(-1j * beta[None, :] * (z1 - zf))).real
    assert np.max(np.abs(y - expect)) <= 1e-11


def test_defocus_broadens_the_lateral_response():
    """Away from the focus the recorded lateral spread grows with |z - z_f|."""
    nx, nz, m = 64, 128, 64
    d = W.geometry(nx, nz, m, na=0.1)
    g = isam.make_geom(d)
    n_f = int(round(d["z_focus_um"] / d["dz_um"]))
    p0 = nx // 2
    p = np.arange(nx) - p0
    widths = []
    for off in (0, 20, 40):
        x = np.zeros((nx, nz), dtype=np.complex128)
        x[p0, n_f + off] = 1.0
        e = np.sum(isam.phi_exact(x, None, g) ** 2, axis=1)
        widths.append(np.sqrt(np.sum(p ** 2 * e) / np.sum(e)))
    assert widths[0] < widths[1] < widths[2]


def test_nufft_matches_exact_ndft():
    """The KB NUFFT (J = 6, sigma = 2, alpha = 2.34 J) against the exact NDFT:
    the relative error stays within the accuracy Fessler & Sutton report for
    this kernel size."""
    g = _geom(64, 256, 256)
    rng = np.random.default_rng(7)
    x = _rand_x(rng, g)
    y = rng.standard_normal((g.nx, g.m))
    mask = W.mask_bernoulli(g.nx, g.m, 0.6, 9)
    ye, yn = isam.phi_exact(x, mask, g), isam.phi_nufft(x, mask, g)
    assert np.linalg.norm(yn - ye) <= 1e-5 * np.linalg.norm(ye)
    xe, xn = isam.phi_adj_exact(y, mask, g), isam.phi_adj_nufft(y, mask, g)
    assert np.linalg.norm(xn - xe) <= 1e-5 * np.linalg.norm(xe)


def test_sampled_direct_sum_matches_full_direct_sum():
    g = _geom(32, 64, 80)
    rng = np.random.default_rng(4)
    x = _rand_x(rng, g)
    full = isam.phi_exact(x, None, g)
    ps = rng.integers(0, g.nx, 25)
    ms = rng.integers(0, g.m, 25)
    assert np.allclose(isam.phi_exact_at(x, g, ps, ms), full[ps, ms], rtol=0, atol=1e-11)


@pytest.mark.parametrize("nu", [0.0, 0.05, 0.125, 0.2, 0.25])
def test_kb_transform_closed_form_matches_quadrature(nu):
    J, alpha = 6, 2.34 * 6
    num, _ = integrate.quad(lambda u: isam.kb_kernel(u, J, alpha) * np.cos(2 * np.pi * u * nu),
                            -J / 2, J / 2, epsabs=0.0, epsrel=1e-13, limit=200)
    assert abs(isam.kb_ft(np.array([nu]), J, alpha)[0] - num) <= 1e-12 * abs(num)


def test_kb_interpolation_reproduces_exponentials():
    """Poisson summation: sum_i psi(t - i) e^{-j 2 pi i nu/K} ~= Psi(nu/K) e^{-j 2 pi t nu/K}
    for |nu| <= K/4: the identity the deapodisation relies on."""
    J, alpha, K = 6, 2.34 * 6, 256
    rng = np.random.default_rng(0)
    worst = 0.0
    for t in rng.uniform(0, K, 50):
        i = np.floor(t - J / 2) + 1 + np.arange(J)
        for nu in np.linspace(-K / 4, K / 4, 33):
            lhs = np.sum(isam.kb_kernel(t - i, J, alpha) * np.exp(-2j * np.pi * i * nu / K))
            rhs = isam.kb_ft(np.array([nu / K]), J, alpha)[0] * np.exp(-2j * np.pi * t * nu / K)
            worst = max(worst, abs(lhs - rhs) / abs(rhs))
    assert worst < 1e-4
