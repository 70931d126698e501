"""FP64 oracle of the ISAM operator for a 3-D volume (Sec. 2.1 with both lateral
axes): the same model as oracle/isam.py with a 2-D lateral Fourier transform.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A volume x[px, py, n] is sampled on a lateral grid dx x dy; its lateral
frequencies are (q_x, q_y) with |q|^2 = q_x^2 + q_y^2, and the ISAM resampling of
Eq. 5 maps depth frequency beta = sqrt(4 k^2 - |q|^2).  Everything else (source,
beam filter G(|q|, k), dispersion phase, focal reference, falloff, real part,
mask) is the B-scan model of oracle/isam.py; a volume with ny = 1 is a B-scan.

    y(p, m) = s(p, m) Re{ ifft2_l[ H(|q_l|, k_m) sum_n w_n X(l, n) e^{-j beta_lm (z_n - z_f)} ] },
    X = fft2 over (px, py) of x.

Two realisations, as for the B-scan: the direct depth sum (phi3_exact and its
transpose) and the Kaiser-Bessel NUFFT of oracle/isam.py applied to every
lateral-frequency row (lx, ly) of the 2-D lateral spectrum (phi3_nufft and its
transpose), which the GPU path is checked against.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import isam

__all__ = ["VolGeom", "make_vol_geom", "lateral_q2", "phi3_exact", "phi3_adj_exact", "phi3_nufft",
           "phi3_adj_nufft"]


@dataclass
class VolGeom:
    g: isam.Geom       # depth, spectrometer, optics and the x axis (nx, dx)
    ny: int
    dy: float


def make_vol_geom(d: dict, ny: int, dy_um: float | None = None) -> VolGeom:
    """A B-scan description plus a second lateral axis of ny pixels (dy = dx by default)."""
    g = isam.make_geom(d)
    return VolGeom(g=g, ny=int(ny), dy=float(dy_um if dy_um is not None else g.dx))


def lateral_q2(v: VolGeom) -> np.ndarray:
    """|q|^2 on the [nx, ny] grid of signed FFT indices."""
    qx = 2.0 * np.pi * np.fft.fftfreq(v.g.nx, d=v.g.dx)
    qy = 2.0 * np.pi * np.fft.fftfreq(v.ny, d=v.dy)
    return qx[:, None] ** 2 + qy[None, :] ** 2


def _beta_filter(v: VolGeom):
    """beta[lx, ly, m] and H[lx, ly, m] (zero where 4 k^2 <= |q|^2)."""
    g = v.g
    q2 = lateral_q2(v)[:, :, None]
    k = g.k[None, None, :]
    b2 = 4.0 * k ** 2 - q2
    prop = b2 > 0.0
    beta = np.sqrt(np.where(prop, b2, 0.0))
    G = np.exp(-q2 / (2.0 * k ** 2 * g.na ** 2)) if g.na > 0 else np.ones_like(b2)
    dk = g.k - g.k0
    omega = g.disp_a * dk ** 2 + g.disp_b * dk ** 3
    H = g.source[None, None, :] * G * np.exp(1j * omega)[None, None, :] * np.exp(-2j * g.k * g.z_f)[None, None, :]
    return beta, np.where(prop, H, 0.0)


def phi3_exact(x: np.ndarray, mask: np.ndarray | None, v: VolGeom) -> np.ndarray:
    """Phi x for a volume x[nx, ny, nz] -> y[nx, ny, m], direct sum over depth."""
    g = v.g
    beta, H = _beta_filter(v)
    w = isam.depth_weight(g)
    z = np.arange(g.nz) * g.dz
    X = np.fft.fft2(np.asarray(x, dtype=np.complex128), axes=(0, 1)) * w[None, None, :]
    U = np.empty((g.nx, v.ny, g.m), dtype=np.complex128)
    for lx in range(g.nx):
        for ly in range(v.ny):
            E = np.exp(-1j * beta[lx, ly][:, None] * (z[None, :] - g.z_f))
            U[lx, ly] = E @ X[lx, ly]
    y = np.fft.ifft2(H * U, axes=(0, 1)).real
    return y if mask is None else y * mask


def phi3_adj_exact(y: np.ndarray, mask: np.ndarray | None, v: VolGeom) -> np.ndarray:
    """The transpose of phi3_exact in the real inner products."""
    g = v.g
    beta, H = _beta_filter(v)
    w = isam.depth_weight(g)
    z = np.arange(g.nz) * g.dz
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    R = np.fft.fft2(r.astype(np.complex128), axes=(0, 1)) / (g.nx * v.ny)
    V = np.conj(H) * R
    W = np.empty((g.nx, v.ny, g.nz), dtype=np.complex128)
    for lx in range(g.nx):
        for ly in range(v.ny):
            E = np.exp(1j * (z[:, None] - g.z_f) * beta[lx, ly][None, :])
            W[lx, ly] = w * (E @ V[lx, ly])
    return (g.nx * v.ny) * np.fft.ifft2(W, axes=(0, 1))


def _kb_position(v: VolGeom, beta: np.ndarray) -> np.ndarray:
    """t = K/(2 pi) (beta dz mod 2 pi) on the K-point axial grid, per (lx, ly, m)."""
    g = v.g
    return np.mod((g.K / (2.0 * np.pi)) * np.mod(beta * g.dz, 2.0 * np.pi), g.K)


def phi3_nufft(x: np.ndarray, mask: np.ndarray | None, v: VolGeom) -> np.ndarray:
    """Phi x for a volume x[nx, ny, nz] with the axial resampling done by the KB
    NUFFT of oracle/isam.py on each of the nx * ny lateral-frequency rows."""
    g = v.g
    beta, H = _beta_filter(v)
    w = isam.depth_weight(g)
    t = _kb_position(v, beta)
    X = np.fft.fft2(np.asarray(x, dtype=np.complex128), axes=(0, 1)) * w[None, None, :]
    U = isam.nufft_axial(X.reshape(g.nx * v.ny, g.nz), t.reshape(g.nx * v.ny, g.m), g).reshape(g.nx, v.ny, g.m)
    U = U * np.exp(1j * beta * (g.z_f - g.n0 * g.dz))
    y = np.fft.ifft2(H * U, axes=(0, 1)).real
    return y if mask is None else y * mask


def phi3_adj_nufft(y: np.ndarray, mask: np.ndarray | None, v: VolGeom) -> np.ndarray:
    """The transpose of phi3_nufft: each of its steps transposed, in reverse order."""
    g = v.g
    beta, H = _beta_filter(v)
    w = isam.depth_weight(g)
    t = _kb_position(v, beta)
    r = np.asarray(y, dtype=np.float64)
    if mask is not None:
        r = r * mask
    R = np.fft.fft2(r.astype(np.complex128), axes=(0, 1)) / (g.nx * v.ny)
    V = np.conj(H) * R * np.exp(-1j * beta * (g.z_f - g.n0 * g.dz))
    a = isam.nufft_axial_adjoint(V.reshape(g.nx * v.ny, g.m), t.reshape(g.nx * v.ny, g.m), g)
    a = a.reshape(g.nx, v.ny, g.nz)
    return (g.nx * v.ny) * np.fft.ifft2(a * w[None, None, :], axes=(0, 1))
