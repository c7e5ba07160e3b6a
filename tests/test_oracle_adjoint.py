"""Pins of the oracle's gradient: the transposes of the TDI and projection operators
(dot-product identity) and the sky-angle derivatives (central finite differences)."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import rel_l2

DT, T0, P = 10.0, 0.0, 11


def setup(N=1500, seed=21):
    src = synth.draw_sources(1, seed=seed, A=1.0)[0]
    orb = synth.orbit_flexing(-2e6, 2e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    return src, o, t0h, hp, hc


@pytest.mark.parametrize("gen", [1, 2])
def test_tdi_adjoint_dot_product(gen):
    _, o, *_ = setup()
    N = 1500
    rng = np.random.default_rng(5)
    y, g = rng.normal(size=(6, N)), rng.normal(size=(3, N))
    lhs = np.sum(oracle.tdi(P, gen, DT, T0, N, o, y) * g)
    rhs = np.sum(y * oracle.tdi_adjoint(P, gen, DT, T0, N, o, g))
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(y * y) * np.sum(g * g))


def test_projection_adjoint_dot_product():
    src, o, t0h, hp, hc = setup()
    N = 1500
    rng = np.random.default_rng(6)
    a, b = rng.normal(size=len(hp)), rng.normal(size=len(hp))
    gy = rng.normal(size=(6, N))
    lhs = np.sum(oracle.project(P, DT, T0, N, o, a, b, t0h, src.lam, src.beta, src.psi) * gy)
    ga, gb = oracle.project_adjoint(P, DT, T0, N, o, len(hp), t0h, src.lam, src.beta, src.psi, gy)
    rhs = np.sum(a * ga) + np.sum(b * gb)
    assert abs(lhs - rhs) < 1e-12 * np.sqrt((np.sum(a * a) + np.sum(b * b)) * np.sum(gy * gy))


def test_strain_gradient_of_quadratic_loss_by_finite_differences():
    """Loss = 1/2 sum (R h - d)^2 is quadratic in h, so the central difference along any
    direction equals the directional derivative up to rounding."""
    src, o, t0h, hp, hc = setup(N=800)
    N = 800
    rng = np.random.default_rng(7)
    d = rng.normal(size=(3, N)) * 1e-3
    R = lambda a, b: oracle.response(P, 2, DT, T0, N, o, o, a, b, t0h, src.lam, src.beta, src.psi)
    loss = lambda a, b: 0.5 * np.sum((R(a, b) - d) ** 2)
    g = R(hp, hc) - d
    ghp, ghc, _ = oracle.backward(P, 2, DT, T0, N, o, o, hp, hc, t0h, src.lam, src.beta, src.psi, g)
    va, vb = rng.normal(size=len(hp)), rng.normal(size=len(hp))
    e = 1e-3
    fd = (loss(hp + e * va, hc + e * vb) - loss(hp - e * va, hc - e * vb)) / (2 * e)
    an = np.sum(ghp * va) + np.sum(ghc * vb)
    assert abs(fd - an) < 1e-8 * abs(an)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_sky_gradient_by_central_differences(which):
    src, o, t0h, hp, hc = setup(N=1000, seed=22)
    N = 1000
    rng = np.random.default_rng(8)
    g = rng.normal(size=(3, N))
    gy = oracle.tdi_adjoint(P, 2, DT, T0, N, o, g)
    an = oracle.sky_gradient(P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi, gy)[which]
    th = np.array([src.lam, src.beta, src.psi])

    def F(v):
        return np.sum(oracle.response(P, 2, DT, T0, N, o, o, hp, hc, t0h, *v) * g)

    # step 1e-4: truncation O(e^2) ~ 1e-8 relative, well above the rounding noise of F
    e = 1e-4 * max(1.0, abs(th[which]))
    tp, tm = th.copy(), th.copy()
    tp[which] += e
    tm[which] -= e
    fd = (F(tp) - F(tm)) / (2 * e)
    assert abs(fd - an) < 1e-6 * abs(an)
