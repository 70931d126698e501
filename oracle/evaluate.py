"""FP64 oracle of the paper's evaluation loop (Sec. 3): the direct ISAM baseline
on linearly interpolated measurements, the normalised cross-correlation of
magnitudes (Eq. ncc) and the golden-section search of lambda.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (it gives no more detail):
  - a missing sample of an A-scan is filled by linear interpolation in the
    spectrometer pixel index between the nearest measured samples on either
    side; before the first and after the last measured sample the nearest
    measured value is held; an A-scan without a measured sample stays zero;
  - "direct ISAM" is the paper's back-projection Phi* (Eq. back_model: the
    Hilbert form, dispersion compensation, resampling, inverse transforms) of the
    interpolated measurements with every sample counted as measured; its scale is
    arbitrary, which the NCC ignores;
  - the lambda search maximises the NCC by golden-section search over
    t = log10(relative lambda) in [lo, hi] with a fixed number of evaluations,
    keeping the best evaluated point (the first one on ties).
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import isam

__all__ = ["interp_measurements", "isam_interpolated", "ncc", "golden_section_max", "INV_PHI"]

INV_PHI = (np.sqrt(5.0) - 1.0) / 2.0


def interp_measurements(y: np.ndarray, mask: np.ndarray | None) -> np.ndarray:
    """Fill the unmeasured samples of every A-scan (row) by linear interpolation in
    the pixel index (np.interp, which holds the end values)."""
    y = np.asarray(y, dtype=np.float64)
    if mask is None:
        return y.copy()
    out = np.zeros_like(y)
    grid = np.arange(y.shape[1], dtype=np.float64)
    for p in range(y.shape[0]):
        idx = np.nonzero(mask[p])[0]
        if idx.size:
            out[p] = np.interp(grid, idx.astype(np.float64), y[p, idx])
    return out


def isam_interpolated(y: np.ndarray, mask: np.ndarray | None, g: isam.Geom) -> np.ndarray:
    """The paper's baseline: direct ISAM (Phi*) of the interpolated measurements."""
    return isam.phi_adj_hilbert_nufft(interp_measurements(y, mask), None, g)


def ncc(x: np.ndarray, z: np.ndarray) -> float:
    """Eq. ncc: correlation of |x| and |z| about their mean magnitudes."""
    a = np.abs(np.asarray(x)).ravel()
    b = np.abs(np.asarray(z)).ravel()
    a = a - a.mean()
    b = b - b.mean()
    return float(np.sum(a * b) / (np.sqrt(np.sum(a * a)) * np.sqrt(np.sum(b * b))))


def golden_section_max(f: Callable[[float], float], lo: float, hi: float, n: int):
    """Golden-section maximisation of f on [lo, hi] with n >= 2 evaluations.

    Interior points c = b - g (b - a) and d = a + g (b - a), g = (sqrt 5 - 1)/2.
    While evaluations remain: if f(c) >= f(d) the maximum is kept in [a, d]
    (b <- d, d <- c, new c), else in [c, b] (a <- c, c <- d, new d).
    Returns (best t, best f, [(t, f) in evaluation order])."""
    a, b = float(lo), float(hi)
    c = b - INV_PHI * (b - a)
    d = a + INV_PHI * (b - a)
    fc, fd = f(c), f(d)
    hist = [(c, fc), (d, fd)]
    while len(hist) < n:
        if fc >= fd:
            b, d, fd = d, c, fc
            c = b - INV_PHI * (b - a)
            fc = f(c)
            hist.append((c, fc))
        else:
            a, c, fc = c, d, fd
            d = a + INV_PHI * (b - a)
            fd = f(d)
            hist.append((d, fd))
    best = max(range(len(hist)), key=lambda i: (hist[i][1], -i))
    return hist[best][0], hist[best][1], hist
