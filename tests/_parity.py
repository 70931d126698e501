"""Parity checks shared by the GPU tests (not a test module).

A single relative L2 over a whole 1024 x 2048 array hides local faults: one
element wrong by ~1 % of the RMS, or one lateral-frequency row (an unpaired row
l = 0 or nx/2 of the paired row kernels, a ragged last column tile) wrong by a
small fraction, barely moves it.  `assert_parity` therefore checks three things:

  - the global relative L2 distance;
  - the relative L2 distance of every lateral-frequency row: the difference and
    the reference are transformed along the lateral axis (a plain numpy FFT of
    both, so a wrong row of the GPU's lateral spectrum shows up undiluted), and
    row l must satisfy |D_l| <= row_tol * max(|R_l|, floor * rms_l |R_l|);
    rows below a quarter of the RMS row (high lateral frequencies that the beam
    filter suppresses) are judged against that quarter instead of their own
    vanishing norm, so that rounding noise spread evenly over the rows passes;
  - the largest element error relative to the RMS of the reference.
"""
from __future__ import annotations

import numpy as np


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def row_errors(got, ref, floor: float = 0.25) -> np.ndarray:
    """Per lateral-frequency row: |FFT_p(got - ref)[l]| / max(|FFT_p(ref)[l]|, floor * RMS row)."""
    d = np.fft.fft(np.asarray(got, dtype=np.complex128) - ref, axis=0)
    r = np.fft.fft(np.asarray(ref, dtype=np.complex128), axis=0)
    dn = np.linalg.norm(d, axis=1)
    rn = np.linalg.norm(r, axis=1)
    rms = np.sqrt(np.mean(rn ** 2))
    return dn / np.maximum(rn, floor * rms)


def max_error(got, ref) -> float:
    """max |got - ref| over the RMS of ref."""
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(got) - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


def assert_parity(got, ref, tol: float, row_tol: float | None = None, max_tol: float | None = None,
                  what: str = "") -> dict:
    """Global relative L2 <= tol, every lateral-frequency row <= row_tol (default
    5 tol), max element error <= max_tol of the RMS (default 20 tol)."""
    row_tol = 5 * tol if row_tol is None else row_tol
    max_tol = 20 * tol if max_tol is None else max_tol
    g = rel_l2(got, ref)
    rows = row_errors(got, ref)
    mx = max_error(got, ref)
    worst = int(np.argmax(rows))
    assert g <= tol, f"{what}: global relative L2 {g:.3e} > {tol:.1e}"
    assert rows[worst] <= row_tol, f"{what}: lateral row {worst} relative L2 {rows[worst]:.3e} > {row_tol:.1e}"
    assert mx <= max_tol, f"{what}: max |error| / RMS {mx:.3e} > {max_tol:.1e}"
    return {"global": g, "row_max": float(rows[worst]), "row_argmax": worst, "max_over_rms": mx}
