"""FP64 oracle of the penalties, proximal maps and the FISTA iteration
(Sec. 2.2-2.3, Eq. alg).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here:
  - spatial sparsity means Psi = I (the text prints "Phi = I");
  - the prox of lambda*||x||_1 over complex x shrinks the modulus:
    z = v * max(0, 1 - tau/|v|), z = 0 where v = 0;
  - the box C of the prox definition is left unconstrained;
  - FISTA starts from x^1 = z^0 = 0, t^1 = 1 and uses delta = 1/(1.01 L) with
    L = lambda_max(Phi^H Phi) from power iteration.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import wavelet

__all__ = ["soft", "prox_l1", "prox_wavelet", "penalty_l1", "penalty_wavelet",
           "objective", "power_iteration", "fista", "ista", "fista_momentum"]

Op = Callable[[np.ndarray], np.ndarray]


def soft(c: np.ndarray, tau: float) -> np.ndarray:
    """Complex soft-threshold: c * max(0, 1 - tau/|c|)."""
    mag = np.abs(c)
    scale = np.where(mag > tau, 1.0 - tau / np.where(mag > 0, mag, 1.0), 0.0)
    return c * scale


def prox_l1(v: np.ndarray, tau: float) -> np.ndarray:
    """prox of tau*||x||_1 (Psi = I, Sec. 2.2)."""
    return soft(v, tau)


def prox_wavelet(v: np.ndarray, tau: float, h: np.ndarray, levels: int = 3) -> np.ndarray:
    """prox of tau*||W x||_1 for orthonormal W: W^T soft(W v, tau)."""
    return wavelet.idwt2(soft(wavelet.dwt2(v, h, levels), tau), h, levels)


def penalty_l1(x: np.ndarray) -> float:
    return float(np.sum(np.abs(x)))


def penalty_wavelet(x: np.ndarray, h: np.ndarray, levels: int = 3) -> float:
    return float(np.sum(np.abs(wavelet.dwt2(x, h, levels))))


def objective(phi: Op, y: np.ndarray, mask: np.ndarray | None, x: np.ndarray,
              lam: float, penalty: Callable[[np.ndarray], float]) -> float:
    """F(x) = 1/2 ||Phi x - s y||^2 + lambda R(x)  (Eqs. obj, ls_obj)."""
    sy = y if mask is None else y * mask
    r = phi(x) - sy
    return 0.5 * float(np.sum(r * r)) + lam * penalty(x)


def power_iteration(phi: Op, phi_adj: Op, shape: tuple, iters: int = 100,
                    seed: int = 0) -> float:
    """Largest eigenvalue of Phi^H Phi (real-linear, on R^{2N}) by power iteration
    from a seeded Gaussian start; the step size bound of Sec. 2.3."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = phi_adj(phi(v))
        lam = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return lam


def fista_momentum(iters: int) -> np.ndarray:
    """mu_k = (t^k - 1)/t^{k+1} for k = 1..iters, t^1 = 1,
    t^{k+1} = (1 + sqrt(1 + 4 (t^k)^2))/2  (Eq. alg)."""
    mu = np.empty(iters)
    t = 1.0
    for k in range(iters):
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        mu[k] = (t - 1.0) / t_next
        t = t_next
    return mu


def fista(phi: Op, phi_adj: Op, y: np.ndarray, mask: np.ndarray | None,
          prox: Callable[[np.ndarray, float], np.ndarray], lam: float, delta: float,
          iters: int, shape: tuple, accelerate: bool = True,
          trace: list | None = None) -> np.ndarray:
    """FISTA (Eq. alg), returning z^iters:

        z^k     = prox_{lambda delta R}(x^k - delta Phi^H(Phi x^k - y))
        t^{k+1} = (1 + sqrt(1 + 4 (t^k)^2)) / 2
        x^{k+1} = z^k + (t^k - 1)/t^{k+1} (z^k - z^{k-1})

    with x^1 = z^0 = 0 and t^1 = 1.  ``accelerate=False`` keeps t = 1 (ISTA).
    ``trace`` collects each z^k when given."""
    sy = y if mask is None else y * mask
    x = np.zeros(shape, dtype=np.complex128)
    z_prev = np.zeros(shape, dtype=np.complex128)
    t = 1.0
    z = z_prev
    for _ in range(iters):
        grad = phi_adj(phi(x) - sy)
        z = prox(x - delta * grad, lam * delta)
        if accelerate:
            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            x = z + ((t - 1.0) / t_next) * (z - z_prev)
            t = t_next
        else:
            x = z
        z_prev = z
        if trace is not None:
            trace.append(z.copy())
    return z


def ista(phi: Op, phi_adj: Op, y: np.ndarray, mask: np.ndarray | None,
         prox: Callable[[np.ndarray, float], np.ndarray], lam: float, delta: float,
         iters: int, shape: tuple, trace: list | None = None) -> np.ndarray:
    """Proximal gradient without momentum (t^k = 1 throughout)."""
    return fista(phi, phi_adj, y, mask, prox, lam, delta, iters, shape, accelerate=False,
                 trace=trace)
