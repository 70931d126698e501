"""Pins of the oracle's proximal maps, step size and FISTA (Sec. 2.3, Eq. alg)."""
import numpy as np
import pytest
from scipy import optimize

from oracle import fista, isam, wavelet
from paper_2108_01438_gb300 import workloads as W


def _tiny_problem(seed=0, mask_keep=0.6):
    g = isam.make_geom(W.geometry(8, 16, 16))
    mask = W.mask_bernoulli(g.nx, g.m, mask_keep, seed + 1)
    x_true = W.point_scatterers(g.nx, g.nz, 5, seed)
    y = isam.phi_exact(x_true, mask, g) + 0.01 * W.unit_noise(g.nx, g.m, seed + 2)
    phi = lambda x: isam.phi_exact(x, mask, g)
    phi_adj = lambda r: isam.phi_adj_exact(r, mask, g)
    return g, mask, y, phi, phi_adj


def _dense(phi, g):
    cols = []
    for part in (1.0, 1j):
        for i in range(g.nx * g.nz):
            e = np.zeros(g.nx * g.nz, dtype=np.complex128)
            e[i] = part
            cols.append(phi(e.reshape(g.nx, g.nz)).ravel())
    return np.array(cols).T


def test_complex_soft_threshold_is_the_prox():
    """Closed form against a numerical minimisation of 1/2|z - v|^2 + tau |z|."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = complex(*rng.standard_normal(2))
        tau = rng.uniform(0.05, 1.5)
        f = lambda u: 0.5 * ((u[0] - v.real) ** 2 + (u[1] - v.imag) ** 2) + tau * np.hypot(u[0], u[1])
        res = optimize.minimize(f, [v.real, v.imag], method="Nelder-Mead",
                                options=dict(xatol=1e-10, fatol=1e-14, maxiter=4000))
        z = fista.soft(np.array([v]), tau)[0]
        assert f([z.real, z.imag]) <= res.fun + 1e-12
        assert abs(z - complex(*res.x)) < 1e-6


def test_wavelet_prox_is_optimal_against_perturbations():
    h = wavelet.daubechies_lowpass(4)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((32, 64)) + 1j * rng.standard_normal((32, 64))
    tau = 0.7
    z = fista.prox_wavelet(v, tau, h)
    obj = lambda x: 0.5 * np.linalg.norm(x - v) ** 2 + tau * fista.penalty_wavelet(x, h)
    f0 = obj(z)
    for _ in range(20):
        d = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)
        assert obj(z + 1e-3 * d) >= f0 - 1e-9


def test_power_iteration_matches_svd():
    g, mask, y, phi, phi_adj = _tiny_problem()
    A = _dense(phi, g)
    smax = np.linalg.svd(A, compute_uv=False)[0]
    L = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=300)
    assert abs(L - smax ** 2) <= 1e-8 * smax ** 2


def test_momentum_sequence():
    mu = fista.fista_momentum(200)
    assert mu[0] == 0.0
    t = 1.0
    for k in range(200):          # t^k >= (k+1)/2, the bound behind the O(1/k^2) rate
        assert t >= (k + 1) / 2 - 1e-12
        t = (1 + np.sqrt(1 + 4 * t * t)) / 2
    assert np.all(np.diff(mu) > 0) and np.all(mu < 1)


def _setup_l1():
    g, mask, y, phi, phi_adj = _tiny_problem()
    L = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=300)
    lam = 0.05 * np.max(np.abs(phi_adj(y * mask)))
    delta = 1.0 / (1.01 * L)
    F = lambda x: fista.objective(phi, y, mask, x, lam, fista.penalty_l1)
    return g, mask, y, phi, phi_adj, L, lam, delta, F


def test_ista_decreases_the_objective_monotonically():
    g, mask, y, phi, phi_adj, L, lam, delta, F = _setup_l1()
    trace = []
    fista.ista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 60, (g.nx, g.nz), trace=trace)
    vals = [F(z) for z in trace]
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(vals, vals[1:]))


def test_fista_rate_bound_and_fixed_point():
    """F(z^k) - F* <= 2 L ||x^1 - x*||^2 / (k+1)^2 (Beck & Teboulle, cited for Eq. alg),
    with F* and x* from a long run whose fixed-point residual vanishes."""
    g, mask, y, phi, phi_adj, L, lam, delta, F = _setup_l1()
    shape = (g.nx, g.nz)
    x_star = fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 4000, shape)
    resid = x_star - fista.prox_l1(x_star - delta * phi_adj(phi(x_star) - y * mask), lam * delta)
    assert np.linalg.norm(resid) <= 1e-6 * np.linalg.norm(x_star)
    f_star = F(x_star)
    trace = []
    fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, delta, 100, shape, trace=trace)
    Lstep = 1.0 / delta
    for k, z in enumerate(trace, start=1):
        assert F(z) - f_star <= 2 * Lstep * np.linalg.norm(x_star) ** 2 / (k + 1) ** 2 + 1e-10


def test_large_lambda_gives_zero():
    """lambda >= max|Phi^H s y| makes 0 a minimiser; FISTA from 0 stays at 0."""
    g, mask, y, phi, phi_adj = _tiny_problem()
    lam = 1.0001 * np.max(np.abs(phi_adj(y * mask)))
    L = fista.power_iteration(phi, phi_adj, (g.nx, g.nz), iters=100)
    z = fista.fista(phi, phi_adj, y, mask, fista.prox_l1, lam, 1 / (1.01 * L), 10, (g.nx, g.nz))
    assert np.all(z == 0)


def test_identity_operator_solves_in_one_step():
    """With Phi = I, delta = 1: the minimiser of 1/2||x - y||^2 + lam ||x||_1 is
    soft(y, lam), reached at the first iterate and kept."""
    rng = np.random.default_rng(5)
    y = rng.standard_normal((4, 6)) + 1j * rng.standard_normal((4, 6))
    ident = lambda x: x
    z = fista.fista(ident, ident, y, None, fista.prox_l1, 0.4, 1.0, 5, y.shape)
    assert np.allclose(z, fista.soft(y, 0.4), atol=1e-15)
