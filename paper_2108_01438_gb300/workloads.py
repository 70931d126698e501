"""Seeded synthetic SD-OCT workloads.

This module only draws random numbers and lays out the optical set-up of a
synthetic experiment (spectrometer grid, source spectrum, beam and dispersion
parameters, phantoms, sub-sampling masks, unit noise).  It holds none of the
reconstruction arithmetic: no system operator, no transform, no solver.  Both
the FP64 oracle and the CUDA path read their inputs from here, so that a parity
check compares the two on identical data.

The paper measured a commercial SD-OCT system (1024 x 1024 A-scans over 4 mm^2,
Sec. 3.1) whose raw data is not available; the phantoms below stand in for the
bead-gel specimen of Sec. 3.1 and the sub-sampling masks follow the random,
equispaced and partial schemes of Sec. 3.1.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2108

__all__ = [
    "BASE_SEED", "spectrometer_k", "geometry", "point_scatterers", "beads",
    "mask_full", "mask_ascans", "mask_bernoulli", "mask_equispaced",
    "mask_partial", "unit_noise", "tiny_workload", "full_workload",
    "smooth_widths", "batch_workload",
]


def spectrometer_k(m: int, lambda_c_um: float = 1.300, bandwidth_um: float = 0.170) -> np.ndarray:
    """Wavenumbers (rad/um) of an m-pixel spectrometer that is linear in wavelength.

    Pixel i sits at lambda_i = lambda_c - bw/2 + i*bw/(m-1); k = 2*pi/lambda, so k
    descends with the pixel index, as on a grating spectrometer.
    """
    lam = lambda_c_um - bandwidth_um / 2 + np.arange(m, dtype=np.float64) * bandwidth_um / (m - 1)
    return 2.0 * np.pi / lam


def geometry(nx: int, nz: int, m: int, *, dx_um: float = 2.0, na: float = 0.1,
             focus_frac: float = 0.5, disp_edge_rad: float = 20.0, disp_b: float = 0.0,
             falloff: bool = True, kb_width: int = 6, kb_oversamp: float = 2.0,
             kb_alpha: float = 0.0, lambda_c_um: float = 1.300,
             bandwidth_um: float = 0.170) -> dict:
    """Optical set-up of one synthetic B-scan as plain numbers.

    - depth pixel dz: the image spans the positive half of the range that the
      spectrometer's largest wavenumber step resolves, dz = pi / (2 nz max|dk|);
    - source spectrum: Gaussian in k, centred mid-span, FWHM half the k-span;
    - focus at ``focus_frac`` of the imaged depth; dispersion a*(k-k0)^2 with ``a``
      set so that the phase reaches ``disp_edge_rad`` at the band edge;
    - falloff half-width twice the imaged depth.
    """
    k = spectrometer_k(m, lambda_c_um, bandwidth_um)
    dk_max = float(np.max(np.abs(np.diff(k))))
    dz = np.pi / (2.0 * nz * dk_max)
    k0 = 0.5 * (k.min() + k.max())
    span = k.max() - k.min()
    fwhm = 0.5 * span
    source = np.exp(-4.0 * np.log(2.0) * ((k - k0) / fwhm) ** 2)
    edge = float(np.max(np.abs(k - k0)))
    return dict(
        nx=int(nx), nz=int(nz), m=int(m), k=k, source=source,
        dx_um=float(dx_um), dz_um=float(dz), na=float(na),
        z_focus_um=float(focus_frac * nz * dz),
        disp_a=float(disp_edge_rad / edge ** 2), disp_b=float(disp_b), k0=float(k0),
        falloff_half_um=float(2.0 * nz * dz) if falloff else 0.0,
        kb_width=int(kb_width), kb_oversamp=float(kb_oversamp), kb_alpha=float(kb_alpha),
    )


def point_scatterers(nx: int, nz: int, count: int, seed: int) -> np.ndarray:
    """``count`` unit-amplitude scatterers with uniform random phase at distinct pixels."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(nx * nz, size=count, replace=False)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=count)
    x = np.zeros(nx * nz, dtype=np.complex128)
    x[flat] = np.exp(1j * phase)
    return x.reshape(nx, nz)


def beads(nx: int, nz: int, count: int, seed: int, background: float = 0.05,
          sigma_px: tuple[float, float] = (1.0, 3.0)) -> np.ndarray:
    """Bead-gel phantom: Gaussian beads (size sigma ~ U[1,3] px, unit amplitude,
    random phase, continuous centres) on a uniform-amplitude random-phase background."""
    rng = np.random.default_rng(seed)
    cp = rng.uniform(0.0, nx, size=count)
    cn = rng.uniform(0.0, nz, size=count)
    sg = rng.uniform(sigma_px[0], sigma_px[1], size=count)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=count)
    bg_phase = rng.uniform(0.0, 2.0 * np.pi, size=(nx, nz))
    x = background * np.exp(1j * bg_phase)
    p = np.arange(nx, dtype=np.float64)
    n = np.arange(nz, dtype=np.float64)
    for b in range(count):
        r = int(np.ceil(4 * sg[b]))
        p_lo, p_hi = max(0, int(cp[b]) - r), min(nx, int(cp[b]) + r + 2)
        n_lo, n_hi = max(0, int(cn[b]) - r), min(nz, int(cn[b]) + r + 2)
        dp = (p[p_lo:p_hi] - cp[b])[:, None]
        dn = (n[n_lo:n_hi] - cn[b])[None, :]
        x[p_lo:p_hi, n_lo:n_hi] += np.exp(1j * ph[b]) * np.exp(-(dp ** 2 + dn ** 2) / (2 * sg[b] ** 2))
    return x


def mask_full(nx: int, m: int) -> np.ndarray:
    return np.ones((nx, m), dtype=np.uint8)


def mask_ascans(nx: int, m: int, keep: float, seed: int) -> np.ndarray:
    """Keep a random ``keep`` fraction of whole A-scans (rows p)."""
    rng = np.random.default_rng(seed)
    kept = rng.choice(nx, size=int(round(keep * nx)), replace=False)
    s = np.zeros((nx, m), dtype=np.uint8)
    s[kept, :] = 1
    return s


def mask_bernoulli(nx: int, m: int, keep: float, seed: int) -> np.ndarray:
    """Per-element Bernoulli(keep) sub-sampling (the 'random' scheme of Sec. 3.1)."""
    rng = np.random.default_rng(seed)
    return (rng.random((nx, m)) < keep).astype(np.uint8)


def mask_equispaced(nx: int, m: int) -> np.ndarray:
    """Every second spectrometer pixel (the 'equispaced' scheme of Sec. 3.1)."""
    s = np.zeros((nx, m), dtype=np.uint8)
    s[:, ::2] = 1
    return s


def mask_partial(nx: int, m: int) -> np.ndarray:
    """The central half of the spectrometer (the 'partial' scheme of Sec. 3.1)."""
    s = np.zeros((nx, m), dtype=np.uint8)
    s[:, m // 4: m // 4 + m // 2] = 1
    return s


def unit_noise(nx: int, m: int, seed: int) -> np.ndarray:
    """Standard normal field; a caller scales it to the SNR it wants."""
    return np.random.default_rng(seed).standard_normal((nx, m))


def smooth_widths(lo: int, hi: int, multiple: int = 8) -> list[int]:
    """Multiples of ``multiple`` in [lo, hi] whose prime factors are all <= 7."""
    out = []
    for w in range(lo, hi + 1):
        if w % multiple:
            continue
        r = w
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        if r == 1:
            out.append(w)
    return out


def tiny_workload(seed_offset: int = 0) -> dict:
    """One 64 x 256 B-scan: 20 point scatterers, full sampling, 30 dB, l1, 50 iterations."""
    seed = BASE_SEED + seed_offset
    nx, nz, m = 64, 256, 256
    return dict(
        name="tiny-64x256-l1", geom=geometry(nx, nz, m), x_true=point_scatterers(nx, nz, 20, seed),
        mask=mask_full(nx, m), noise=unit_noise(nx, m, seed + 1000), snr_db=30.0,
        penalty="l1", lambda_frac=0.01, iters=50,
    )


def full_workload(seed_offset: int = 1) -> dict:
    """One 1024 x 2048 B-scan: 500 beads, half the A-scans, 25 dB, db4 3-level, 100 iterations."""
    seed = BASE_SEED + seed_offset
    nx, nz, m = 1024, 2048, 2048
    return dict(
        name="full-1024x2048-db4", geom=geometry(nx, nz, m), x_true=beads(nx, nz, 500, seed),
        mask=mask_ascans(nx, m, 0.5, seed + 7), noise=unit_noise(nx, m, seed + 1000), snr_db=25.0,
        penalty="db4", lambda_frac=0.01, iters=100,
    )


def batch_workload(count: int = 64, seed_offset: int = 2, widths: tuple[int, int] = (256, 2048),
                   depths: tuple[int, ...] = (1024, 2048), scatterers: int = 200) -> list[dict]:
    """Uneven batch: widths drawn uniformly from the 7-smooth multiples of 8 in
    ``widths``, depth (= spectral pixels) from ``depths``, per-scan focus depth
    U[0.25, 0.75] of the imaged depth and dispersion up to 30 rad at the band edge,
    per-element Bernoulli sub-sampling keeping U[0.25, 0.75] of the samples,
    point-scatterer phantoms, l1, 100 iterations."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    choices = smooth_widths(*widths)
    out = []
    for i in range(count):
        nx = int(rng.choice(choices))
        nz = int(rng.choice(depths))
        m = nz
        focus = float(rng.uniform(0.25, 0.75))
        a_edge = float(rng.uniform(-30.0, 30.0))
        b_edge = float(rng.uniform(-10.0, 10.0))
        keep = float(rng.uniform(0.25, 0.75))
        d = geometry(nx, nz, m, focus_frac=focus, disp_edge_rad=a_edge)
        edge = float(np.max(np.abs(d["k"] - d["k0"])))
        d["disp_b"] = b_edge / edge ** 3
        s = int(rng.integers(1 << 30))
        out.append(dict(
            name=f"batch-{i}-{nx}x{nz}", geom=d, x_true=point_scatterers(nx, nz, scatterers, s),
            mask=mask_bernoulli(nx, m, keep, s + 1), noise=unit_noise(nx, m, s + 2), snr_db=30.0,
            penalty="l1", lambda_frac=0.01, iters=100,
        ))
    return out
