"""FP64 oracle of the ISAM system operator Phi and its adjoint (Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
library, shares no code with the CUDA path.

Notation (all lengths in micrometres, wavenumbers in rad/um):
  x[p, n]   complex image, p = A-scan (lateral pixel dx), n = depth pixel (dz),
            z_n = n*dz, zero delay at n = 0.
  y[p, m]   real spectrometer samples at wavenumber k_m; s[p, m] in {0, 1} the
            sub-sampling mask (Eq. for_model, diag(s)).
  q_l       lateral spatial frequency 2*pi*l~/(nx*dx), l~ the signed FFT index.
  beta_lm   axial object frequency sqrt(4 k_m^2 - q_l^2): the ISAM resampling
            k = sqrt(beta^2 + q^2)/2 of Eq. 5 solved for beta.

The forward model written out (Eq. for_model, with the readings below):

  y(p,m) = s(p,m) Re{ (1/nx) sum_l e^{+j 2 pi l p/nx} H_lm
                       sum_n w_n X(l,n) e^{-j beta_lm (z_n - z_f)} },
  X(l,n) = sum_p x(p,n) e^{-j 2 pi l p/nx}                 (lateral FT, Eq. 4)
  H_lm   = A(k_m) G(q_l,k_m) e^{j Omega(k_m)} e^{-j 2 k_m z_f}

  - Omega = a (k-k0)^2 + b (k-k0)^3 is the dispersion phase of Sec. 2.1;
  - G = exp(-q^2 / (2 k^2 NA^2)) is the ISAM filter f^ (Eq. 5), which the paper
    leaves unspecified: a double-pass Gaussian beam whose focus sits at depth
    z_f, so that the in-focus plane carries no lateral blur;
  - A(k) is the source spectrum and w_n = exp(-ln2 (z_n/z_half)^2) the
    depth falloff named in the abstract;
  - the zero-padding Q and the DFT D of Eq. for_model are absorbed by evaluating
    the axial transform directly at the spectrometer wavenumbers, with the image
    confined to the positive half of the unambiguous depth range.
The adjoint used is the exact transpose of Phi in the real inner products
<a,b> = Re sum conj(a) b, i.e. Phi^H y = B^H (s * y) with y embedded as y + 0j.

The paper's own back-projection (Eq. back_model) is given too:
  Phi*(y) = B^H A(s * y),  A(r) = r - j d H(r)   (phi_adj_hilbert_*)
with H the discrete Hilbert transform along the spectrometer axis (the DFT
multiplier -j sgn(f), zero at DC and at the Nyquist bin).  Readings: the printed
order "K^H D^H Q^T" is taken as K^H Q^T D^H (the only order whose sizes agree),
and d = +1 when k increases with the pixel index (A = Re - jH, as printed) and
d = -1 when it decreases (A = Re + jH): A keeps the side of the spectrum on which
e^{-j 2 k z}, z > 0, lies, so that A(Re{w}) = w for such a signal w.  On those
signals Phi* = 2 Phi^H on the image the twin cannot reach: the conjugate (twin)
term of the transpose is dropped and the kept term is doubled.

Two realisations are given:
  phi_exact / phi_adj_exact  - a direct non-uniform DFT over depth.
  phi_nufft / phi_adj_nufft  - the Kaiser-Bessel NUFFT (Fessler & Sutton) that
                               the paper uses to realise the resampling (Sec. 2.1,
                               "u = Kx"): deapodise, zero-pad to K = sigma*nz,
                               FFT, interpolate J taps.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft
from scipy.special import i0

__all__ = [
    "Geom", "make_geom", "lateral_q", "axial_beta", "system_filter", "depth_weight",
    "kb_kernel", "kb_ft", "kb_grid_position", "phi_exact", "phi_adj_exact",
    "phi_exact_at", "phi_nufft", "phi_adj_nufft", "nufft_axial", "nufft_axial_adjoint",
    "b_adj_exact", "b_adj_nufft", "hilbert", "conj_analytic", "k_increasing",
    "phi_adj_hilbert_exact", "phi_adj_hilbert_nufft", "phi_qd",
]


@dataclass
class Geom:
    nx: int
    nz: int
    m: int
    k: np.ndarray
    source: np.ndarray
    dx: float
    dz: float
    na: float
    z_f: float
    disp_a: float
    disp_b: float
    k0: float
    z_half: float
    J: int
    sigma: float
    alpha: float

    @property
    def K(self) -> int:
        """Oversampled axial grid size sigma*nz."""
        return int(round(self.sigma * self.nz))

    @property
    def n0(self) -> int:
        """Depth index about which the NUFFT phase is centred."""
        return self.nz // 2


def make_geom(d: dict) -> Geom:
    """Geometry from the plain-number description of a workload.

    dz = 0 selects pi/(2 nz max|dk|): the positive, twin-free half of the depth
    range the spectrometer resolves.  kb_alpha = 0 selects alpha = 2.34 J, the
    Kaiser-Bessel shape Fessler & Sutton recommend for sigma = 2.
    """
    k = np.asarray(d["k"], dtype=np.float64)
    nz = int(d["nz"])
    dz = float(d.get("dz_um", 0.0))
    if dz <= 0:
        dz = np.pi / (2.0 * nz * np.max(np.abs(np.diff(k))))
    src = d.get("source")
    src = np.ones_like(k) if src is None else np.asarray(src, dtype=np.float64)
    J = int(d.get("kb_width", 6))
    alpha = float(d.get("kb_alpha", 0.0)) or 2.34 * J
    return Geom(nx=int(d["nx"]), nz=nz, m=int(d["m"]), k=k, source=src,
                dx=float(d["dx_um"]), dz=dz, na=float(d.get("na", 0.0)),
                z_f=float(d.get("z_focus_um", 0.0)), disp_a=float(d.get("disp_a", 0.0)),
                disp_b=float(d.get("disp_b", 0.0)), k0=float(d.get("k0", 0.0)),
                z_half=float(d.get("falloff_half_um", 0.0)), J=J,
                sigma=float(d.get("kb_oversamp", 2.0)), alpha=alpha)


# ---------------------------------------------------------------- geometry

def lateral_q(g: Geom) -> np.ndarray:
    """q_l = 2 pi l~ / (nx dx) with l~ the signed FFT index (Eq. 4, lateral axis)."""
    return 2.0 * np.pi * np.fft.fftfreq(g.nx, d=g.dx)


def axial_beta(g: Geom) -> tuple[np.ndarray, np.ndarray]:
    """beta_lm = sqrt(4 k_m^2 - q_l^2) (Eq. 5) and the mask of propagating (l, m)."""
    q = lateral_q(g)
    b2 = 4.0 * g.k[None, :] ** 2 - q[:, None] ** 2
    prop = b2 > 0.0
    return np.sqrt(np.where(prop, b2, 0.0)), prop


def system_filter(g: Geom) -> np.ndarray:
    """H_lm = A(k) G(q,k) e^{j Omega(k)} e^{-j 2 k z_f}: source, ISAM beam filter
    (Eq. 5), dispersion phase (Sec. 2.1) and the focal-plane phase reference."""
    q = lateral_q(g)
    _, prop = axial_beta(g)
    k = g.k[None, :]
    if g.na > 0:
        G = np.exp(-q[:, None] ** 2 / (2.0 * k ** 2 * g.na ** 2))
    else:
        G = np.ones((g.nx, g.m))
    dk = g.k - g.k0
    omega = g.disp_a * dk ** 2 + g.disp_b * dk ** 3
    H = g.source[None, :] * G * np.exp(1j * omega)[None, :] * np.exp(-2j * g.k * g.z_f)[None, :]
    return np.where(prop, H, 0.0)


def depth_weight(g: Geom) -> np.ndarray:
    """Falloff w(z_n) = exp(-ln2 (z_n / z_half)^2); 1 when z_half <= 0."""
    z = np.arange(g.nz) * g.dz
    if g.z_half <= 0:
        return np.ones(g.nz)
    return np.exp(-np.log(2.0) * (z / g.z_half) ** 2)


# ------------------------------------------------------- direct (exact) NDFT

def phi_exact(x: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi x by a direct sum over depth (no NUFFT): O(nx m nz)."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    z = np.arange(g.nz) * g.dz
    X = np.fft.fft(np.asarray(x, dtype=np.complex128), axis=0)
    a = X * w[None, :]
    U = np.empty((g.nx, g.m), dtype=np.complex128)
    for l in range(g.nx):
        E = np.exp(-1j * beta[l][:, None] * (z[None, :] - g.z_f))
        U[l] = E @ a[l]
    y = np.fft.ifft(H * U, axis=0).real
    return y if mask is None else y * mask


def phi_exact_at(x: np.ndarray, g: Geom, ps: np.ndarray, ms: np.ndarray) -> np.ndarray:
    """Unmasked (Phi x)(p, m) at the listed samples, each by a direct sum."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    z = np.arange(g.nz) * g.dz
    a = np.fft.fft(np.asarray(x, dtype=np.complex128), axis=0) * w[None, :]
    lat = np.arange(g.nx)
    out = np.empty(len(ps))
    for mm in np.unique(ms):
        E = np.exp(-1j * beta[:, mm][:, None] * (z[None, :] - g.z_f))
        U = np.sum(a * E, axis=1) * H[:, mm]
        for i in np.nonzero(ms == mm)[0]:
            out[i] = (np.sum(np.exp(2j * np.pi * lat * ps[i] / g.nx) * U) / g.nx).real
    return out


def phi_adj_exact(y: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi^H y, the transpose of phi_exact in the real inner products."""
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    return b_adj_exact(r.astype(np.complex128), g)


def b_adj_exact(c: np.ndarray, g: Geom) -> np.ndarray:
    """B^H c for a complex measurement-domain array c[p, m], B the complex-valued
    forward map before the real part (direct sum over depth)."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    z = np.arange(g.nz) * g.dz
    R = np.fft.fft(np.asarray(c, dtype=np.complex128), axis=0) / g.nx
    V = np.conj(H) * R
    W = np.empty((g.nx, g.nz), dtype=np.complex128)
    for l in range(g.nx):
        E = np.exp(1j * (z[:, None] - g.z_f) * beta[l][None, :])
        W[l] = w * (E @ V[l])
    return g.nx * np.fft.ifft(W, axis=0)


# ------------------------------------------------------ Kaiser-Bessel NUFFT
#
# The NUFFT path runs on every host core: its FFTs through scipy.fft with one
# worker per core, and its per-row steps (deapodise, pad, axial FFT, interpolate
# or spread) on blocks of rows in threads.  Rows never interact in those steps,
# so a block's arithmetic is the same as the whole array's, element by element.

WORKERS = max(1, os.cpu_count() or 1)


def _fft(a, axis):
    return sfft.fft(a, axis=axis, workers=WORKERS)


def _ifft(a, axis):
    return sfft.ifft(a, axis=axis, workers=WORKERS)


def _by_rows(fn, *arrays):
    """fn(*arrays) evaluated on blocks of rows (axis 0) in threads, concatenated."""
    n = arrays[0].shape[0]
    nb = min(WORKERS, n)
    if nb <= 1 or arrays[0].size < (1 << 15):
        return fn(*arrays)
    cut = np.linspace(0, n, nb + 1).astype(int)
    with ThreadPoolExecutor(nb) as ex:
        parts = list(ex.map(lambda b: fn(*(a[cut[b]:cut[b + 1]] for a in arrays)), range(nb)))
    return np.concatenate(parts, axis=0)


def kb_kernel(u: np.ndarray, J: int, alpha: float) -> np.ndarray:
    """psi(u) = I0(alpha sqrt(1 - (2u/J)^2)) / I0(alpha) on |u| <= J/2, else 0."""
    u = np.asarray(u, dtype=np.float64)
    r = 1.0 - (2.0 * u / J) ** 2
    inside = r >= 0.0
    return np.where(inside, i0(alpha * np.sqrt(np.where(inside, r, 0.0))) / i0(alpha), 0.0)


def kb_ft(nu: np.ndarray, J: int, alpha: float) -> np.ndarray:
    """Fourier transform of psi at frequency nu (cycles per grid cell):

        Psi(nu) = J sinh(sqrt(alpha^2 - (pi J nu)^2)) / sqrt(alpha^2 - (pi J nu)^2) / I0(alpha)

    (the sin form where pi J |nu| > alpha)."""
    nu = np.asarray(nu, dtype=np.float64)
    s2 = alpha ** 2 - (np.pi * J * nu) ** 2
    out = np.empty_like(nu)
    pos = s2 > 1e-30
    neg = s2 < -1e-30
    mid = ~(pos | neg)
    sp = np.sqrt(s2[pos])
    out[pos] = np.sinh(sp) / sp
    sn = np.sqrt(-s2[neg])
    out[neg] = np.sin(sn) / sn
    out[mid] = 1.0
    return J * out / i0(alpha)


def kb_grid_position(g: Geom) -> np.ndarray:
    """t_lm = K/(2 pi) * (beta_lm dz mod 2 pi), the position of frequency beta_lm dz
    on the K-point axial grid."""
    beta, _ = axial_beta(g)
    t = (g.K / (2.0 * np.pi)) * np.mod(beta * g.dz, 2.0 * np.pi)
    return np.mod(t, g.K)


def nufft_axial(a: np.ndarray, t: np.ndarray, g: Geom) -> np.ndarray:
    """Rows a[l, n] -> sum_n a[l,n] e^{-j omega_lm (n - n0)} at omega = 2 pi t/K,
    approximated by the Kaiser-Bessel NUFFT of Fessler & Sutton:
      1. deapodise: b_n = a_n / Psi((n - n0)/K)
      2. zero-pad to K with the index centred at n0 and take a K-point FFT
      3. interpolate with J taps i = floor(t - J/2) + 1 + j, weights psi(t - i)."""
    return _by_rows(lambda a_, t_: _nufft_axial_rows(a_, t_, g), a, t)


def _nufft_axial_rows(a: np.ndarray, t: np.ndarray, g: Geom) -> np.ndarray:
    K, J = g.K, g.J
    n = np.arange(g.nz)
    b = a / kb_ft((n - g.n0) / K, J, g.alpha)[None, :]
    pad = np.zeros((a.shape[0], K), dtype=np.complex128)
    pad[:, (n - g.n0) % K] = b
    Y = sfft.fft(pad, axis=1)
    base = np.floor(t - J / 2.0).astype(np.int64) + 1
    rows = np.arange(a.shape[0])[:, None]
    U = np.zeros(t.shape, dtype=np.complex128)
    for j in range(J):
        i = base + j
        U += kb_kernel(t - i, J, g.alpha) * Y[rows, i % K]
    return U


def nufft_axial_adjoint(V: np.ndarray, t: np.ndarray, g: Geom) -> np.ndarray:
    """Transpose of nufft_axial: spread each V[l,m] onto its J grid taps, take the
    unnormalised inverse K-point FFT, keep the nz centred samples, deapodise."""
    return _by_rows(lambda v_, t_: _nufft_axial_adjoint_rows(v_, t_, g), V, t)


def _nufft_axial_adjoint_rows(V: np.ndarray, t: np.ndarray, g: Geom) -> np.ndarray:
    K, J = g.K, g.J
    rows_n = V.shape[0]
    base = np.floor(t - J / 2.0).astype(np.int64) + 1
    rows = np.broadcast_to(np.arange(rows_n)[:, None], t.shape)
    Gk = np.zeros(rows_n * K, dtype=np.complex128)
    for j in range(J):
        i = base + j
        contrib = kb_kernel(t - i, J, g.alpha) * V
        flat = (rows * K + i % K).ravel()
        Gk += np.bincount(flat, weights=contrib.real.ravel(), minlength=rows_n * K)
        Gk += 1j * np.bincount(flat, weights=contrib.imag.ravel(), minlength=rows_n * K)
    Yb = K * sfft.ifft(Gk.reshape(rows_n, K), axis=1)
    n = np.arange(g.nz)
    b = Yb[:, (n - g.n0) % K]
    return b / kb_ft((n - g.n0) / K, J, g.alpha)[None, :]


def phi_nufft(x: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi x with the axial resampling done by the KB NUFFT (the paper's K of
    Sec. 2.1).  The NUFFT evaluates the depth sum centred on z_c = n0 dz; the
    factor e^{j beta (z_f - z_c)} moves the phase reference to the focus."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    t = kb_grid_position(g)
    X = _fft(np.asarray(x, dtype=np.complex128), 0)
    U = nufft_axial(X * w[None, :], t, g)
    U = U * np.exp(1j * beta * (g.z_f - g.n0 * g.dz))
    y = _ifft(H * U, 0).real
    return y if mask is None else y * mask


def phi_adj_nufft(y: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi^H y for phi_nufft: the transpose of each of its steps, in reverse order."""
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    return b_adj_nufft(r.astype(np.complex128), g)


def b_adj_nufft(c: np.ndarray, g: Geom) -> np.ndarray:
    """B^H c with the KB NUFFT, for a complex measurement-domain array c[p, m]."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    t = kb_grid_position(g)
    R = _fft(np.asarray(c, dtype=np.complex128), 0) / g.nx
    V = np.conj(H) * R * np.exp(-1j * beta * (g.z_f - g.n0 * g.dz))
    a = nufft_axial_adjoint(V, t, g)
    return g.nx * _ifft(a * w[None, :], 0)


# ------------------------------------------- Hilbert-form back-projection

def hilbert(r: np.ndarray) -> np.ndarray:
    """Discrete Hilbert transform of real r along its last axis: the DFT
    multiplier -j sgn(f), with f the signed frequency index and sgn = 0 at DC and,
    for even lengths, at the Nyquist bin."""
    r = np.asarray(r, dtype=np.float64)
    M = r.shape[-1]
    f = np.arange(M)
    sgn = np.where((f > 0) & (2 * f < M), 1.0, np.where(2 * f > M, -1.0, 0.0))
    return np.fft.ifft(-1j * sgn * np.fft.fft(r, axis=-1), axis=-1).real


def conj_analytic(r: np.ndarray, d: int = 1) -> np.ndarray:
    """A(r) = r - j d H(r) of Eq. back_model (d = +1 as printed, the conjugate
    analytic signal; d = -1 its mirror for a descending wavenumber axis)."""
    r = np.asarray(r, dtype=np.float64)
    return r - 1j * d * hilbert(r)


def k_increasing(g: Geom) -> bool:
    return bool(g.k[-1] > g.k[0])


def _hilbert_side(g: Geom) -> int:
    return 1 if k_increasing(g) else -1


def phi_adj_hilbert_exact(y: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """The paper's back-projection Phi*(y) = B^H A(s y) (Eq. back_model), direct sum."""
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    return b_adj_exact(conj_analytic(r, _hilbert_side(g)), g)


def phi_adj_hilbert_nufft(y: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi*(y) = B^H A(s y) (Eq. back_model) with the KB NUFFT."""
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    return b_adj_nufft(conj_analytic(r, _hilbert_side(g)), g)


# ------------------------------------------------ literal Q and D of Eq. for_model

def phi_qd(x: np.ndarray, mask: np.ndarray | None, g: Geom) -> np.ndarray:
    """Phi x through the literal steps of Eq. for_model: per lateral frequency the
    weighted depth profile is zero-padded to P = 2 nz (Q) and transformed by a
    P-point DFT (D); the ISAM resampling (K) then reads the profile's spectrum at
    theta = beta dz from those P samples by band-limited (Dirichlet) interpolation,
        A(theta) = (1/P) sum_i S_i sum_{n<P} e^{j (2 pi i/P - theta) n},
    which is exact because the profile vanishes on the padding.  The inner sum
    is the closed-form geometric series."""
    beta, _ = axial_beta(g)
    H = system_filter(g)
    w = depth_weight(g)
    P = 2 * g.nz
    X = np.fft.fft(np.asarray(x, dtype=np.complex128), axis=0) * w[None, :]
    S = np.fft.fft(np.concatenate([X, np.zeros_like(X)], axis=1), axis=1)      # D Q
    i = np.arange(P)
    U = np.empty((g.nx, g.m), dtype=np.complex128)
    for l in range(g.nx):
        theta = beta[l] * g.dz
        phi = 2.0 * np.pi * i[None, :] / P - theta[:, None]
        den = 1.0 - np.exp(1j * phi)
        num = 1.0 - np.exp(-1j * theta[:, None] * P)
        on_grid = np.abs(den) < 1e-12
        ker = np.where(on_grid, P, num / np.where(on_grid, 1.0, den))
        U[l] = (ker @ S[l]) / P
    U = U * np.exp(1j * beta * g.z_f)
    y = np.fft.ifft(H * U, axis=0).real
    return y if mask is None else y * mask
