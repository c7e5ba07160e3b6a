"""Pins of the oracle's rounding-error scales (the `absval` evaluations that size the parity
tolerances: every weight, coefficient and input by its absolute value).  They must bound the
magnitude of the plain evaluation term by term (triangle inequality), depend on the inputs only
through their absolute values, and scale linearly with them."""
import numpy as np
import pytest

import oracle
import synth

DT, T0, P, N = 10.0, 0.0, 11, 600


@pytest.fixture(scope="module")
def setup():
    orb = synth.orbit_flexing(-2e6, 2e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    src = synth.draw_sources(1, seed=2, A=1e-21, fdot=1e-17)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    return o, src, t0h, hp, hc


def test_projection_scale(setup):
    o, src, t0h, hp, hc = setup
    args = (P, DT, T0, N, o)
    ang = (t0h, src.lam, src.beta, src.psi)
    y = oracle.project(*args, hp, hc, *ang)
    e = oracle.project(*args, hp, hc, *ang, absval=True)
    assert np.all(e >= np.abs(y) * (1 - 1e-12))
    np.testing.assert_allclose(oracle.project(*args, -hp, np.abs(hc), *ang, absval=True), e, rtol=1e-14)
    np.testing.assert_allclose(oracle.project(*args, 3 * hp, 3 * hc, *ang, absval=True), 3 * e, rtol=1e-14)


@pytest.mark.parametrize("gen", [1, 2])
def test_tdi_scale(setup, gen):
    o = setup[0]
    y = np.random.default_rng(gen).normal(size=(6, N))
    x = oracle.tdi(P, gen, DT, T0, N, o, y)
    e = oracle.tdi(P, gen, DT, T0, N, o, y, absval=True)
    assert np.all(e >= np.abs(x) * (1 - 1e-12))
    np.testing.assert_allclose(oracle.tdi(P, gen, DT, T0, N, o, -np.abs(y), absval=True), e, rtol=1e-14)
    np.testing.assert_allclose(oracle.tdi(P, gen, DT, T0, N, o, 0.5 * y, absval=True), 0.5 * e, rtol=1e-14)


def test_sky_gradient_scale(setup):
    o, src, t0h, hp, hc = setup
    gy = np.random.default_rng(7).normal(size=(6, N))
    args = (P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    g = oracle.sky_gradient(*args, gy)
    e = oracle.sky_gradient(*args, gy, absval=True)
    assert np.all(e >= np.abs(g) * (1 - 1e-12))
    np.testing.assert_allclose(oracle.sky_gradient(*args, -gy, absval=True), e, rtol=1e-14)
