"""Pins of the oracle's projection onto the six links (Sec. "Projection on the constellation
arms": antenna patterns and Eq. instrument-response-to-gw; Sec. "Reference frames")."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import C, LINKS, k_vector, rel_l2, relabel_positions, constant_orbit_from

DT, T0, P = 10.0, 0.0, 25
L_STATIC = 2.5e9 / C


def static_orbit():
    o = synth.orbit_static(-2e6, 2e6)
    return o, oracle.Orbit(o.t_knots, o.pos, o.delays)


def linear_patterns(lam, beta, psi, orb_o, n_out=300):
    """xi+ and xix of each link read off the response to h+ = t and hx = t.  For a static
    triangle with L = |x_r - x_s|/c the exact response to a linear strain is -(L/2) xi
    (the interpolation is exact for polynomials)."""
    t0h = T0 - 80 * DT
    t = t0h + DT * np.arange(n_out + 160) - 1500.0
    z = np.zeros_like(t)
    yp = oracle.project(P, DT, T0, n_out, orb_o, t, z, t0h, lam, beta, psi)
    yc = oracle.project(P, DT, T0, n_out, orb_o, z, t, t0h, lam, beta, psi)
    return -2.0 * yp[:, 150] / L_STATIC, -2.0 * yc[:, 150] / L_STATIC, yp, yc


def test_linear_strain_response_is_constant_minus_half_L_xi():
    orb, o = static_orbit()
    xp, xc, yp, yc = linear_patterns(1.0, 0.3, 0.4, o)
    # constant in time (static geometry)
    assert np.max(np.abs(yp[:, 100:200] - yp[:, 150:151])) < 1e-12 * np.abs(yp).max()
    # pattern identity: xi+^2 + xix^2 = (1 - (k.n)^2)^2 for every link
    k = k_vector(1.0, 0.3)
    x = orb.pos[:, :, 0]
    for l, (r, s) in enumerate(LINKS):
        n = (x[r - 1] - x[s - 1]) / np.linalg.norm(x[r - 1] - x[s - 1])
        assert abs(xp[l] ** 2 + xc[l] ** 2 - (1 - np.dot(k, n) ** 2) ** 2) < 1e-12
    # patterns are even in n: a link and its reverse agree
    for a, b in [(0, 5), (1, 4), (2, 3)]:
        assert abs(xp[a] - xp[b]) < 1e-12 and abs(xc[a] - xc[b]) < 1e-12


def test_polarisation_angle_rotates_patterns():
    orb, o = static_orbit()
    xp0, xc0, *_ = linear_patterns(0.7, -0.4, 0.0, o)
    xp1, xc1, *_ = linear_patterns(0.7, -0.4, np.pi / 4, o)
    xp2, xc2, *_ = linear_patterns(0.7, -0.4, np.pi / 2, o)
    assert np.allclose(xp1, xc0, atol=1e-12) and np.allclose(xc1, -xp0, atol=1e-12)
    assert np.allclose(xp2, -xp0, atol=1e-12) and np.allclose(xc2, -xc0, atol=1e-12)


def test_ecliptic_pole_source_on_in_plane_arm():
    """Hand-derived special case: for beta = pi/2 and an arm along (cos a, sin a, 0),
    u.n = sin(lam - a) and v.n = -cos(lam - a), so xi+ = -cos 2(lam - a), xix = -sin 2(lam - a)."""
    a = 0.83
    x1 = np.array([synth.AU, 0.0, 0.0])
    x2 = x1 - 2.5e9 * np.array([np.cos(a), np.sin(a), 0.0])
    x3 = x1 - 2.5e9 * np.array([np.cos(a + np.pi / 3), np.sin(a + np.pi / 3), 0.0])
    tk, pos, dl = constant_orbit_from(np.stack([x1, x2, x3]), np.full(6, L_STATIC), -2e6, 2e6)
    o = oracle.Orbit(tk, pos, dl)
    for lam in [0.0, 0.4, 2.9]:
        xp, xc, *_ = linear_patterns(lam, np.pi / 2, 0.0, o)
        assert abs(xp[0] - (-np.cos(2 * (lam - a)))) < 1e-9
        assert abs(xc[0] - (-np.sin(2 * (lam - a)))) < 1e-9


def test_source_normal_to_constellation_plane():
    """k perpendicular to every arm: xi+^2 + xix^2 = 1, and the three arms (120 degrees
    apart, patterns periodic in 2 x angle) sum to zero."""
    orb, o = static_orbit()
    nrm = np.array([-np.sin(np.pi / 3), 0.0, np.cos(np.pi / 3)])
    beta = np.arcsin(-nrm[2])
    lam = np.arctan2(-nrm[1], -nrm[0])
    assert np.allclose(k_vector(lam, beta), nrm)
    xp, xc, *_ = linear_patterns(lam, beta, 0.3, o)
    assert np.allclose(xp ** 2 + xc ** 2, 1.0, atol=1e-12)
    assert abs(xp[:3].sum()) < 1e-12 and abs(xc[:3].sum()) < 1e-12


def analytic_y(src, orb, xp, xc, lam, beta, t):
    """y from the closed-form strain at the exact emission and reception times of a
    static triangle; the patterns are those read off the linear-strain response."""
    k = k_vector(lam, beta)
    x = orb.pos[:, :, 0]
    out = np.empty((6, len(t)))
    for l, (r, s) in enumerate(LINKS):
        n = (x[r - 1] - x[s - 1]) / np.linalg.norm(x[r - 1] - x[s - 1])
        te = t - L_STATIC - np.dot(k, x[s - 1]) / C
        tr = t - np.dot(k, x[r - 1]) / C
        hpe, hce = synth.gb_polarisations(src, te)
        hpr, hcr = synth.gb_polarisations(src, tr)
        out[l] = (xp[l] * (hpe - hpr) + xc[l] * (hce - hcr)) / (2 * (1 - np.dot(k, n)))
    return out


def test_sinusoid_matches_closed_form_static_triangle():
    src = synth.config1_source()
    orb, o = static_orbit()
    xp, xc, *_ = linear_patterns(src.lam, src.beta, src.psi, o)
    N = 4096
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    y = oracle.project(P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    ya = analytic_y(src, orb, xp, xc, src.lam, src.beta, synth.sample_grid(T0, DT, N))
    assert rel_l2(y, ya) < 1e-12


def test_low_frequency_limit_is_minus_half_L_strain_derivative():
    """For f L << 1, y_l -> -(L/2) dH_l/dt, taken midway between the emission-time read
    (t - L - k.x_s/c) and the reception-time read (t - k.x_r/c = t - L - k.x_s/c + L(1 - k.n));
    the relative deviation is O((2 pi f L)^2)."""
    src = synth.Source(A=1.0, f=2e-6, fdot=0.0, phi0=0.3, iota=0.9, psi=0.2, lam=2.0, beta=-0.5, fddot=0.0)
    orb, o = static_orbit()
    xp, xc, *_ = linear_patterns(src.lam, src.beta, src.psi, o)
    N = 600
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    y = oracle.project(P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    t = synth.sample_grid(T0, DT, N)
    k = k_vector(src.lam, src.beta)
    d = 1e-3
    x = orb.pos[:, :, 0]
    for l, (r, s) in enumerate(LINKS):
        n = (x[r - 1] - x[s - 1]) / np.linalg.norm(x[r - 1] - x[s - 1])
        te = t - L_STATIC - np.dot(k, x[s - 1]) / C + 0.5 * L_STATIC * (1 - np.dot(k, n))
        p1, c1 = synth.gb_polarisations(src, te + d)
        p0, c0 = synth.gb_polarisations(src, te - d)
        dH = (xp[l] * (p1 - p0) + xc[l] * (c1 - c0)) / (2 * d)
        ylf = -0.5 * L_STATIC * dH
        assert rel_l2(y[l, 100:500], ylf[100:500]) < 1e-6


def test_geometry_is_evaluated_at_the_output_time():
    """On a moving orbit, y at sample n equals y of a rigid constellation frozen at the
    positions and delays of time t_n."""
    src = synth.draw_sources(1, seed=11, A=1e-21)[0]
    orb = synth.orbit_flexing(-2e6, 6e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    N = 400000
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    for n in [1000, 123456, 398000]:
        yn = oracle.project_at(P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi, [n])[:, 0]
        pos, dl = o.eval(T0 + n * DT)
        tk, fpos, fdl = constant_orbit_from(pos, dl, -2e6, 6e6)
        of = oracle.Orbit(tk, fpos, fdl)
        yf = oracle.project_at(P, DT, T0, N, of, hp, hc, t0h, src.lam, src.beta, src.psi, [n])[:, 0]
        assert np.max(np.abs(yn - yf)) <= 1e-11 * np.max(np.abs(yn))


def test_linearity_and_zero():
    src = synth.config1_source()
    orb, o = static_orbit()
    N = 2048
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    r1 = synth.random_series(len(hp), 1, 1e-21)
    r2 = synth.random_series(len(hp), 2, 1e-21)
    a, b = 0.37, -1.9
    f = lambda u, v: oracle.project(P, DT, T0, N, o, u, v, t0h, src.lam, src.beta, src.psi)
    lhs = f(a * hp + b * r1, a * hc + b * r2)
    rhs = a * f(hp, hc) + b * f(r1, r2)
    assert rel_l2(lhs, rhs) < 1e-13
    z = np.zeros_like(hp)
    assert not np.any(f(z, z))


def test_cyclic_relabelling_of_spacecraft_permutes_links():
    """Relabel x'_i = x_sigma(i), sigma = (1->2, 2->3, 3->1): y'_ij = y_sigma(i)sigma(j)."""
    src = synth.draw_sources(1, seed=12, A=1e-21)[0]
    orb = synth.orbit_flexing(-2e6, 3e6)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    o2 = oracle.Orbit(orb.t_knots, relabel_positions(orb.pos, [1, 2, 0]), None)
    N = 8192
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    y = oracle.project(P, DT, T0, N, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    y2 = oracle.project(P, DT, T0, N, o2, hp, hc, t0h, src.lam, src.beta, src.psi)
    sig = {1: 2, 2: 3, 3: 1}
    for l, (r, s) in enumerate(LINKS):
        l2 = LINKS.index((sig[r], sig[s]))
        assert np.max(np.abs(y2[l] - y[l2])) <= 1e-13 * np.abs(y).max()
