"""FP64 oracle of the isotropic total-variation penalty (Sec. 2.2) and its
proximal map (Sec. 2.3, the prox of Eq. alg with R = TV).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The penalty, as the paper writes it for a complex image x[i, j]:

    TV(x) = sum_{i,j} sqrt(|x(i+1,j) - x(i,j)|^2 + |x(i,j+1) - x(i,j)|^2)

Readings of the paper used here (it is silent on these points):
  - a difference that would leave the image is zero (the last row has no
    lateral difference and the last column no depth difference);
  - prox_{tau TV}(v) = argmin_x 1/2 ||x - v||^2 + tau TV(x) is computed by the
    fast gradient projection on the dual problem (Beck and Teboulle's FGP for
    isotropic TV denoising), a fixed number of iterations, starting from the zero
    dual at every call;
  - the dual variable p = (p1, p2) holds one complex number per direction and
    pixel and is feasible when |p1|^2 + |p2|^2 <= 1 at every pixel.

With grad x = (d1, d2), d1 = x(i+1,j) - x(i,j), d2 = x(i,j+1) - x(i,j) (zero at the
far edges), TV(x) = max_{p feasible} Re <grad x, p> = max_p -Re <x, div p>, where
div = -grad^T.  Hence the prox is x = v + tau div p* with p* minimising
1/2 ||v + tau div p||^2 over feasible p, a smooth problem whose gradient
-tau grad(v + tau div p) has Lipschitz constant at most 8 tau^2.
"""
from __future__ import annotations

import numpy as np

__all__ = ["grad", "div", "tv", "project", "prox_tv", "dual_gap"]


def grad(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Forward differences along both axes, zero where they would leave the image."""
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    d1[:-1, :] = x[1:, :] - x[:-1, :]
    d2[:, :-1] = x[:, 1:] - x[:, :-1]
    return d1, d2


def div(p1: np.ndarray, p2: np.ndarray) -> np.ndarray:
    """div = -grad^T, written out: the backward differences of p, where p1 on the
    last row and p2 on the last column take no part (grad never fills them)."""
    P, N = p1.shape
    out = np.zeros_like(p1)
    out[:-1, :] += p1[:-1, :]
    out[1:, :] -= p1[:-1, :]
    out[:, :-1] += p2[:, :-1]
    out[:, 1:] -= p2[:, :-1]
    return out


def tv(x: np.ndarray) -> float:
    """TV(x) of Sec. 2.2 (complex moduli, isotropic over the two directions)."""
    d1, d2 = grad(x)
    return float(np.sum(np.sqrt(np.abs(d1) ** 2 + np.abs(d2) ** 2)))


def project(p1: np.ndarray, p2: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Pixelwise projection onto |p1|^2 + |p2|^2 <= 1."""
    nrm = np.sqrt(np.abs(p1) ** 2 + np.abs(p2) ** 2)
    s = 1.0 / np.maximum(1.0, nrm)
    return p1 * s, p2 * s


def prox_tv(v: np.ndarray, tau: float, iters: int = 20, return_dual: bool = False):
    """prox_{tau TV}(v) by `iters` FGP steps on the dual from p = 0.

    Step k (t_1 = 1, r_1 = p_0 = 0):
        p_k     = project(r_k + grad(v + tau div r_k) / (8 tau))
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        r_{k+1} = p_k + (t_k - 1)/t_{k+1} (p_k - p_{k-1})
    and the result is x = v + tau div p_iters.
    """
    v = np.asarray(v, dtype=np.complex128)
    if tau <= 0 or iters <= 0:
        return (v.copy(), np.zeros_like(v), np.zeros_like(v)) if return_dual else v.copy()
    p1 = np.zeros_like(v)
    p2 = np.zeros_like(v)
    q1, q2 = p1.copy(), p2.copy()          # p_{k-1}
    r1, r2 = p1.copy(), p2.copy()
    t = 1.0
    for _ in range(iters):
        g1, g2 = grad(v + tau * div(r1, r2))
        p1, p2 = project(r1 + g1 / (8.0 * tau), r2 + g2 / (8.0 * tau))
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        m = (t - 1.0) / tn
        r1, r2 = p1 + m * (p1 - q1), p2 + m * (p2 - q2)
        q1, q2 = p1, p2
        t = tn
    x = v + tau * div(p1, p2)
    return (x, p1, p2) if return_dual else x


def fgp_momentum(iters: int) -> np.ndarray:
    """(t_k - 1)/t_{k+1} for k = 1 .. iters, the momentum after step k."""
    out = np.zeros(iters)
    t = 1.0
    for k in range(iters):
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        out[k] = (t - 1.0) / tn
        t = tn
    return out


def dual_gap(v: np.ndarray, tau: float, p1: np.ndarray, p2: np.ndarray) -> float:
    """Primal minus dual objective at x = v + tau div p for a feasible p:
    P(x) = 1/2 ||x - v||^2 + tau TV(x),  D(p) = 1/2 ||v||^2 - 1/2 ||v + tau div p||^2.
    Weak duality makes it non-negative; it is zero exactly at the prox."""
    x = v + tau * div(p1, p2)
    primal = 0.5 * np.sum(np.abs(x - v) ** 2) + tau * tv(x)
    dual = 0.5 * np.sum(np.abs(v) ** 2) - 0.5 * np.sum(np.abs(x) ** 2)
    return float(primal - dual)
