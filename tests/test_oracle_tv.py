"""Pins of the TV oracle (oracle/tv.py) to facts that do not come from it: the
adjoint identity of its difference operators, closed-form TV values, and an
optimality certificate of its prox (the duality gap, zero only at the minimiser
by weak duality), plus special cases that reduce to known answers."""
import numpy as np
import pytest

from oracle import tv

RNG = np.random.default_rng(2108)


def _c(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


def test_div_is_minus_grad_transpose():
    """Re<grad x, p> = -Re<x, div p> for random complex x, p (a dropped term, a
    wrong sign or a transposed index in either operator breaks it)."""
    for shape in [(7, 5), (1, 9), (9, 1), (16, 32)]:
        x, p1, p2 = _c(shape), _c(shape), _c(shape)
        d1, d2 = tv.grad(x)
        lhs = np.real(np.vdot(d1, p1) + np.vdot(d2, p2))
        rhs = -np.real(np.vdot(x, tv.div(p1, p2)))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0), shape


def test_tv_closed_forms():
    P, N = 6, 9
    assert tv.tv(np.full((P, N), 3.0 - 2.0j)) == 0.0
    # a step of complex height h across the lateral axis: one difference per column
    h = 2.0 + 1.5j
    x = np.zeros((P, N), complex)
    x[3:, :] = h
    assert abs(tv.tv(x) - N * abs(h)) <= 1e-12
    # the same step along depth: one difference per row
    y = np.zeros((P, N), complex)
    y[:, 4:] = h
    assert abs(tv.tv(y) - P * abs(h)) <= 1e-12
    # a single interior impulse of height a: sqrt(2)|a| at the pixel itself (both
    # differences leave it), |a| at its upper and left neighbours
    a = 1.0 - 2.0j
    z = np.zeros((P, N), complex)
    z[2, 3] = a
    assert abs(tv.tv(z) - (np.sqrt(2.0) + 2.0) * abs(a)) <= 1e-12
    # a linear ramp x(i, j) = alpha i + beta j: interior pixels see sqrt(|alpha|^2 + |beta|^2)
    alpha, beta = 0.3 + 0.1j, -0.2 + 0.4j
    i, j = np.meshgrid(np.arange(P), np.arange(N), indexing="ij")
    r = alpha * i + beta * j
    want = ((P - 1) * (N - 1) * np.sqrt(abs(alpha) ** 2 + abs(beta) ** 2)
            + (N - 1) * abs(beta) + (P - 1) * abs(alpha))
    assert abs(tv.tv(r) - want) <= 1e-10


def test_projection_is_onto_the_unit_ball():
    p1, p2 = 3 * _c((8, 8)), 3 * _c((8, 8))
    q1, q2 = tv.project(p1, p2)
    nrm = np.sqrt(np.abs(q1) ** 2 + np.abs(q2) ** 2)
    assert np.all(nrm <= 1 + 1e-12)
    inside = np.sqrt(np.abs(p1) ** 2 + np.abs(p2) ** 2) <= 1
    assert np.array_equal(q1[inside], p1[inside])


@pytest.mark.parametrize("shape,tau", [((12, 16), 0.3), ((9, 7), 1.0), ((1, 24), 0.5)])
def test_prox_reaches_the_minimiser(shape, tau):
    """The duality gap of the FGP pair goes to zero (and is never negative): an
    optimality certificate that does not use the iteration itself."""
    v = _c(shape)
    gaps = []
    for it in (5, 50, 2000):
        x, p1, p2 = tv.prox_tv(v, tau, it, return_dual=True)
        assert np.all(np.sqrt(np.abs(p1) ** 2 + np.abs(p2) ** 2) <= 1 + 1e-12)
        g = tv.dual_gap(v, tau, p1, p2)
        assert g >= -1e-9
        gaps.append(g)
    assert gaps[2] <= 1e-6 * (0.5 * np.sum(np.abs(v) ** 2))
    assert gaps[2] <= gaps[0]


def test_prox_special_cases():
    v = _c((10, 12))
    # tau = 0: identity
    assert np.array_equal(tv.prox_tv(v, 0.0), v)
    # a constant image is its own prox (TV = 0 and the quadratic is zero there)
    c = np.full((10, 12), 0.7 - 0.2j)
    assert np.max(np.abs(tv.prox_tv(c, 5.0, 50) - c)) <= 1e-12
    # the mean is preserved (div p sums to zero)
    x = tv.prox_tv(v, 0.8, 100)
    assert abs(np.mean(x) - np.mean(v)) <= 1e-12
    # a huge tau flattens the image to its mean
    xf = tv.prox_tv(v, 1e3, 3000)
    assert np.max(np.abs(xf - np.mean(v))) <= 1e-3 * np.max(np.abs(v))


def test_prox_of_a_two_level_signal_has_the_textbook_shrinkage():
    """1 x N real signal with a single step of height h between two plateaus of
    length n: for tau < n h / 2 the prox moves each plateau towards the other by
    tau / n (the jump shrinks by 2 tau / n) and stays piecewise constant."""
    n, h, tau = 8, 2.0, 1.5
    v = np.concatenate([np.zeros(n), np.full(n, h)])[None, :].astype(complex)
    x = tv.prox_tv(v, tau, 5000)
    want = np.concatenate([np.full(n, tau / n), np.full(n, h - tau / n)])[None, :]
    assert np.max(np.abs(x - want)) <= 1e-6
