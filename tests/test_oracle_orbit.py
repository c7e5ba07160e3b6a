"""Pins of the oracle's orbit handling: cubic-spline interpolation of spacecraft positions
and delays (Sec. "Implementation": orbital information interpolated to the sample grid) and
the Newtonian light-time solve used when delays are not supplied."""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline

import oracle
import synth

C = synth.C_LIGHT


@pytest.mark.parametrize("uniform", [True, False])
def test_spline_reproduces_cubics_not_a_knot(uniform):
    rng = np.random.default_rng(5)
    tk = np.linspace(0, 10, 12) if uniform else np.sort(rng.uniform(0, 10, 12))
    f = lambda t: 0.3 * t ** 3 - 2 * t ** 2 + t - 4
    t = rng.uniform(tk[0] - 0.5, tk[-1] + 0.5, 50)
    got = oracle.spline_eval(tk, f(tk), t, oracle.NOT_A_KNOT)
    assert np.max(np.abs(got - f(t))) < 1e-11 * np.max(np.abs(f(t)))


@pytest.mark.parametrize("bc,name", [(oracle.NOT_A_KNOT, "not-a-knot"), (oracle.NATURAL, "natural")])
def test_spline_matches_scipy(bc, name):
    rng = np.random.default_rng(6)
    tk = np.sort(rng.uniform(0, 100, 30))
    y = rng.normal(size=30)
    t = rng.uniform(tk[0], tk[-1], 200)
    ref = CubicSpline(tk, y, bc_type=name)(t)
    got = oracle.spline_eval(tk, y, t, bc)
    assert np.max(np.abs(got - ref)) < 1e-12 * (1 + np.abs(ref).max())
    assert np.max(np.abs(oracle.spline_eval(tk, y, tk, bc) - y)) < 1e-13


def test_static_triangle_constant_and_exact():
    orb = synth.orbit_static(-1e6, 1e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    for t in [-3.3e5, 0.0, 12345.6, 9.9e5]:
        pos, d = o.eval(t)
        assert np.array_equal(d, np.full(6, 2.5e9 / C))
        assert np.allclose(pos, orb.pos[:, :, 0], rtol=0, atol=1e-4)
    # the printed static arm: 2.5e9 m / c = 8.3391023800 s
    assert abs(2.5e9 / C - 8.3391023800) < 1e-10


def test_light_time_static_equals_distance_over_c():
    orb = synth.orbit_static(-1e6, 1e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    d = o.delays_at_knots()
    assert np.max(np.abs(d - 2.5e9 / C)) < 1e-12


def test_light_time_moving_orbit_solves_the_equation():
    orb = synth.orbit_equal_arm(0, 3.2e7)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    d = o.delays_at_knots()
    # residual of | x_r(t) - x_s(t - L) | = c L at a few knots (positions from scipy's spline)
    sp = [[CubicSpline(orb.t_knots, orb.pos[i, c], bc_type="not-a-knot") for c in range(3)] for i in range(3)]
    links = [(0, 1), (1, 2), (2, 0), (0, 2), (2, 1), (1, 0)]
    for k in [3, 100, 250]:
        t = orb.t_knots[k]
        for l, (r, s) in enumerate(links):
            L = d[l, k]
            xr = np.array([sp[r][c](t) for c in range(3)])
            xs = np.array([sp[s][c](t - L) for c in range(3)])
            assert abs(np.linalg.norm(xr - xs) / C - L) < 1e-12
    # moving spacecraft: the two directions of an arm differ (Sagnac-like), by ~1e-4..1e-2 s,
    # and an equal-arm constellation keeps each delay within ~1e-3 s of its mean
    assert 1e-5 < np.max(np.abs(d[0] - d[5])) < 1e-2
    assert np.max(np.ptp(d, axis=1)) < 5e-3


def test_flexing_orbit_arms_flex_one_percent():
    orb = synth.orbit_flexing(0, 3.2e7)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    d = o.delays_at_knots()
    rel = d / (2.5e9 / C) - 1.0
    assert 0.008 < np.max(np.abs(rel)) < 0.012
