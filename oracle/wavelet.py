"""FP64 oracle of the orthonormal wavelet penalty transform Psi (Sec. 2.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's wavelet penalty is the dual-tree complex wavelet; the reconstruction
here uses an orthonormal Daubechies wavelet with 4 vanishing moments (8 taps),
3 levels, periodic boundaries, applied separably over both image axes and to the
real and imaginary parts alike.  With an orthonormal Psi the proximal map of
lambda ||Psi x||_1 is Psi^T soft(Psi v) in closed form.

The filter is derived, not tabulated: Daubechies' construction takes the
low-pass response H(w) = ((1 + e^{-jw})/2)^N L(w) with
|L(w)|^2 = P(sin^2(w/2)), P(u) = sum_{k<N} C(N-1+k, k) u^k, and factors P
spectrally, keeping the roots inside the unit circle (minimum phase).
"""
from __future__ import annotations

from math import comb

import numpy as np

__all__ = ["daubechies_lowpass", "quadrature_mirror", "dwt1_level", "idwt1_level",
           "dwt2", "idwt2"]


def daubechies_lowpass(vanishing: int = 4) -> np.ndarray:
    """Minimum-phase Daubechies low-pass filter h[0..2N-1], sum h = sqrt(2).

    With u = sin^2(w/2) = (2 - z - 1/z)/4, z^{N-1} P(u(z)) is a degree-2(N-1)
    polynomial whose roots come in reciprocal pairs; the ones inside the unit
    circle become the zeros of L.  h, read as the coefficients of
    h0 z^{2N-1} + ... + h_{2N-1}, has N zeros at z = -1 and those roots.
    """
    N = vanishing
    # P(u) with u = (2 - z - z^-1)/4, multiplied by z^{N-1}: a Laurent expansion.
    # u * z = (-z^2 + 2z - 1)/4 as a polynomial in z (highest power first).
    uz = np.array([-0.25, 0.5, -0.25])
    poly = np.zeros(2 * (N - 1) + 1)
    for kk in range(N):
        term = np.array([1.0])
        for _ in range(kk):
            term = np.polymul(term, uz)
        # term has degree 2kk and stands for u^kk z^kk; lift it to z^{N-1}
        shifted = np.concatenate([np.zeros(N - 1 - kk), term, np.zeros(N - 1 - kk)])
        poly = poly + comb(N - 1 + kk, kk) * shifted
    roots = np.roots(poly)
    inside = roots[np.abs(roots) < 1.0]
    h = np.real(np.poly(np.concatenate([-np.ones(N), inside])))
    return h * (np.sqrt(2.0) / np.sum(h))


def quadrature_mirror(h: np.ndarray) -> np.ndarray:
    """High-pass g_n = (-1)^n h_{L-1-n}."""
    L = len(h)
    return np.array([(-1) ** n * h[L - 1 - n] for n in range(L)])


def dwt1_level(x: np.ndarray, h: np.ndarray, axis: int) -> tuple[np.ndarray, np.ndarray]:
    """One periodic analysis level along ``axis``:
    a_k = sum_i h_i x[(2k+i) mod n],  d_k = sum_i g_i x[(2k+i) mod n]."""
    g = quadrature_mirror(h)
    x = np.moveaxis(x, axis, 0)
    n = x.shape[0]
    a = np.zeros((n // 2,) + x.shape[1:], dtype=x.dtype)
    d = np.zeros_like(a)
    for kk in range(n // 2):
        for i in range(len(h)):
            a[kk] += h[i] * x[(2 * kk + i) % n]
            d[kk] += g[i] * x[(2 * kk + i) % n]
    return np.moveaxis(a, 0, axis), np.moveaxis(d, 0, axis)


def idwt1_level(a: np.ndarray, d: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """Transpose (= inverse) of dwt1_level: x[(2k+i) mod n] += h_i a_k + g_i d_k."""
    g = quadrature_mirror(h)
    a = np.moveaxis(a, axis, 0)
    d = np.moveaxis(d, axis, 0)
    n = 2 * a.shape[0]
    x = np.zeros((n,) + a.shape[1:], dtype=np.result_type(a, d))
    for kk in range(n // 2):
        for i in range(len(h)):
            x[(2 * kk + i) % n] += h[i] * a[kk] + g[i] * d[kk]
    return np.moveaxis(x, 0, axis)


def dwt2(x: np.ndarray, h: np.ndarray, levels: int = 3) -> np.ndarray:
    """Separable periodic 2-D analysis, Mallat layout: at each level the current
    low-low block [0:P, 0:N] becomes [[LL, LH], [HL, HH]] with the first index the
    lateral axis p and the second the depth axis n (L/H = low/high along p, then n)."""
    c = np.array(x, dtype=np.result_type(x, np.float64), copy=True)
    P, N = c.shape
    for _ in range(levels):
        blk = c[:P, :N]
        lo_n, hi_n = dwt1_level(blk, h, axis=1)
        ll, hl = dwt1_level(lo_n, h, axis=0)
        lh, hh = dwt1_level(hi_n, h, axis=0)
        c[:P // 2, :N // 2] = ll
        c[:P // 2, N // 2:N] = lh
        c[P // 2:P, :N // 2] = hl
        c[P // 2:P, N // 2:N] = hh
        P, N = P // 2, N // 2
    return c


def idwt2(c: np.ndarray, h: np.ndarray, levels: int = 3) -> np.ndarray:
    """Inverse of dwt2 (its transpose, the transform being orthonormal)."""
    x = np.array(c, copy=True)
    P0, N0 = x.shape
    for lev in reversed(range(levels)):
        P, N = P0 >> lev, N0 >> lev
        ll = x[:P // 2, :N // 2]
        lh = x[:P // 2, N // 2:N]
        hl = x[P // 2:P, :N // 2]
        hh = x[P // 2:P, N // 2:N]
        lo_n = idwt1_level(ll, hl, h, axis=0)
        hi_n = idwt1_level(lh, hh, h, axis=0)
        x[:P, :N] = idwt1_level(lo_n, hi_n, h, axis=1)
    return x
