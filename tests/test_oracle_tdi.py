"""Pins of the oracle's second-generation TDI (Sec. "Time-delay interferometry",
Eqs. tdi1 and tdi2, chained delays as sums; Y, Z by cyclic permutation)."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import C, LINKS, LINK_INDEX, rel_l2, relabel_positions, constant_orbit_from

DT, T0, P = 10.0, 0.0, 25
SIG = {1: 2, 2: 3, 3: 1}


def perm_link(name, times):
    r, s = int(name[0]), int(name[1])
    for _ in range(times):
        r, s = SIG[r], SIG[s]
    return f"{r}{s}"


def phasor_closed_form(c, L, omega, gen):
    """X1 = (1 - D12 D21)(y13 + D13 y31) - (1 - D13 D31)(y12 + D12 y21) and
    X2 = (1 - D13 D31 D12 D21) X1 for constant delays (operators commute), derived by hand
    from Eqs. tdi1/tdi2; D_ij -> exp(-i omega L_ij) on y_ij = Re(c_ij exp(i omega t)).
    Returns the complex amplitudes of X, Y, Z."""
    out = []
    for ch in range(3):
        nm = lambda s: perm_link(s, ch)
        D = lambda s: np.exp(-1j * omega * L[LINK_INDEX[nm(s)]])
        y = lambda s: c[LINK_INDEX[nm(s)]]
        A = D("13") * D("31")
        B = D("12") * D("21")
        x1 = (1 - B) * (y("13") + D("13") * y("31")) - (1 - A) * (y("12") + D("12") * y("21"))
        out.append(x1 if gen == 1 else (1 - A * B) * x1)
    return np.array(out)


def const_delay_orbit(L6):
    pos = synth.static_triangle(np.zeros(1))[:, :, 0]
    tk, pp, dl = constant_orbit_from(pos, L6, -2e6, 2e6)
    return oracle.Orbit(tk, pp, dl)


L_UNEQUAL = np.array([8.10, 8.25, 8.40, 8.20, 8.35, 8.05])


@pytest.mark.parametrize("gen", [1, 2])
def test_constant_unequal_arms_match_phasor_closed_form(gen):
    rng = np.random.default_rng(3)
    c = rng.normal(size=6) + 1j * rng.normal(size=6)
    omega = 2 * np.pi * 4e-3
    N = 1024
    t = synth.sample_grid(T0, DT, N)
    y = np.real(c[:, None] * np.exp(1j * omega * t)[None, :])
    o = const_delay_orbit(L_UNEQUAL)
    xyz = oracle.tdi(P, gen, DT, T0, N, o, y)
    ref = np.real(phasor_closed_form(c, L_UNEQUAL, omega, gen)[:, None] * np.exp(1j * omega * t)[None, :])
    sl = slice(40, N - 20)   # away from the zero-extended ends
    assert rel_l2(xyz[:, sl], ref[:, sl]) < 1e-11


def test_integer_delays_are_exact_shifted_sums():
    """With delays that are whole samples the reads are exact, and X2 equals the operator
    form applied with integer shifts."""
    dt = 1.0
    Lint = np.array([8, 9, 7, 6, 10, 5])
    rng = np.random.default_rng(4)
    N = 400
    y = rng.normal(size=(6, N))
    o = const_delay_orbit(Lint.astype(float))
    xyz = oracle.tdi(P, 2, dt, T0, N, o, y)

    def shift(v, k):
        out = np.zeros_like(v)
        out[k:] = v[:len(v) - k]
        return out

    for ch in range(3):
        nm = lambda s: perm_link(s, ch)
        S = lambda s: (lambda v: shift(v, int(Lint[LINK_INDEX[nm(s)]])))
        Y = lambda s: y[LINK_INDEX[nm(s)]]
        A = lambda v: S("13")(S("31")(v))
        B = lambda v: S("12")(S("21")(v))
        u = Y("13") + S("13")(Y("31"))
        w = Y("12") + S("12")(Y("21"))
        x1 = (u - B(u)) - (w - A(w))
        x2 = x1 - A(B(x1))
        sl = slice(60, N - 20)
        assert np.max(np.abs(xyz[ch, sl] - x2[sl])) < 1e-13 * np.abs(x2).max()


def flexing_delays():
    orb = synth.orbit_flexing(-2e6, 3.3e7)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    return orb, o


def test_delays_are_all_taken_at_the_output_time():
    """Summed chained delays: X at sample n equals X computed with every delay frozen at its
    value at t_n."""
    orb, o = flexing_delays()
    rng = np.random.default_rng(8)
    N = 3000
    y = rng.normal(size=(6, N))
    xyz = oracle.tdi(P, 2, DT, T0, N, o, y)
    for n in [500, 1777, 2900]:
        _, dl = o.eval(T0 + n * DT)
        of = const_delay_orbit(dl)
        xf = oracle.tdi(P, 2, DT, T0, N, of, y)
        assert np.max(np.abs(xf[:, n] - xyz[:, n])) < 1e-12 * np.abs(xyz[:, n]).max()


def test_mirror_delays_and_links_cancel_exactly():
    """With L12 = L13 and L21 = L31 (time-varying) and y12 = y13, y21 = y31, every term of
    X1 and X2 meets a partner of opposite sign and an identical read: X vanishes to the
    rounding of the running sum."""
    orb, o = flexing_delays()
    d = o.delays_at_knots()
    d[LINK_INDEX["13"]] = d[LINK_INDEX["12"]]
    d[LINK_INDEX["31"]] = d[LINK_INDEX["21"]]
    om = oracle.Orbit(orb.t_knots, orb.pos, d)
    rng = np.random.default_rng(9)
    N = 2000
    y = rng.normal(size=(6, N))
    y[LINK_INDEX["13"]] = y[LINK_INDEX["12"]]
    y[LINK_INDEX["31"]] = y[LINK_INDEX["21"]]
    for gen in (1, 2):
        x = oracle.tdi(P, gen, DT, T0, N, om, y)
        assert np.max(np.abs(x[0])) < 1e-14 * np.abs(y).max()
        assert np.abs(x[1]).max() > 0.1 and np.abs(x[2]).max() > 0.1


def test_X_ignores_the_links_and_delays_it_does_not_contain():
    orb, o = flexing_delays()
    rng = np.random.default_rng(10)
    N = 1500
    y = rng.normal(size=(6, N))
    x = oracle.tdi(P, 2, DT, T0, N, o, y)
    y2 = y.copy()
    y2[LINK_INDEX["23"]] += 1.0
    y2[LINK_INDEX["32"]] -= 2.0
    d = o.delays_at_knots()
    d[LINK_INDEX["23"]] += 0.3
    d[LINK_INDEX["32"]] -= 0.2
    x2 = oracle.tdi(P, 2, DT, T0, N, oracle.Orbit(orb.t_knots, orb.pos, d), y2)
    assert np.array_equal(x[0], x2[0])
    assert not np.array_equal(x[1], x2[1])


def test_cyclic_and_reflection_symmetry_on_flexing_orbits():
    """Relabelling spacecraft by sigma = (1->2->3->1) maps (X, Y, Z) -> (Y, Z, X); the
    reflection 2 <-> 3 maps X -> -X and Y <-> -Z (the equations are unchanged up to sign)."""
    src = synth.draw_sources(1, seed=13, A=1e-21)[0]
    orb = synth.orbit_flexing(-2e6, 3e6)
    N = 6000
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    args = (P, 2, DT, T0, N)

    def run(pos):
        o = oracle.Orbit(orb.t_knots, pos, None)
        return oracle.response(*args, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)

    x = run(orb.pos)
    xc = run(relabel_positions(orb.pos, [1, 2, 0]))
    xr = run(relabel_positions(orb.pos, [0, 2, 1]))
    s = np.abs(x).max()
    assert np.max(np.abs(xc[0] - x[1])) <= 1e-13 * s
    assert np.max(np.abs(xc[1] - x[2])) <= 1e-13 * s
    assert np.max(np.abs(xc[2] - x[0])) <= 1e-13 * s
    assert np.max(np.abs(xr[0] + x[0])) <= 1e-13 * s
    assert np.max(np.abs(xr[1] + x[2])) <= 1e-13 * s
    assert np.max(np.abs(xr[2] + x[1])) <= 1e-13 * s


def test_nested_equals_summed_for_constant_delays_and_differs_otherwise():
    rng = np.random.default_rng(12)
    N = 1200
    y = rng.normal(size=(6, N))
    oc = const_delay_orbit(L_UNEQUAL)
    a = oracle.tdi(P, 2, DT, T0, N, oc, y, oracle.DELAY_SUM)
    b = oracle.tdi(P, 2, DT, T0, N, oc, y, oracle.DELAY_NESTED)
    assert rel_l2(b, a) < 1e-12   # nested form subtracts times of size t: rounding of t
    orb, o = flexing_delays()
    a = oracle.tdi(P, 2, DT, T0, N, o, y, oracle.DELAY_SUM)
    b = oracle.tdi(P, 2, DT, T0, N, o, y, oracle.DELAY_NESTED)
    assert 0 < rel_l2(b, a) < 1e-3


def test_equal_arm_transfer_magnitude():
    """Equal constant arms L, y13 - y12 with everything else zero: |X2| = |1 - D^2| |1 - D^4|
    |c13 - c12| = 4 |sin(omega L)| |sin(2 omega L)| |c13 - c12|."""
    omega = 2 * np.pi * 7e-3
    L = 2.5e9 / C
    c = np.zeros(6, complex)
    c[LINK_INDEX["13"]] = 1.0 + 0.5j
    c[LINK_INDEX["12"]] = -0.3 + 0.2j
    N = 2048
    t = synth.sample_grid(T0, DT, N)
    y = np.real(c[:, None] * np.exp(1j * omega * t)[None, :])
    x = oracle.tdi(P, 2, DT, T0, N, const_delay_orbit(np.full(6, L)), y)
    amp = np.abs(np.fft.rfft(x[0, 100:100 + 1800] * np.hanning(1800))).max()
    amp0 = np.abs(np.fft.rfft(np.cos(omega * t[100:1900]) * np.hanning(1800))).max()
    expect = 4 * abs(np.sin(omega * L)) * abs(np.sin(2 * omega * L)) * abs(c[3] - c[0])
    assert abs(amp / amp0 - expect) < 1e-3 * expect


@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("mode", ["summed", "nested"])
def test_quadratic_links_reduce_tdi_to_its_chained_delays(gen, mode):
    """With every link series the parabola y(t) = (t / 100 s)^2 (read exactly by the Lagrange FIR,
    degree 2 <= p) and delays linear in time (reproduced exactly by the cubic spline), each delayed
    term is y(t - D) for its chained delay D, so X follows by hand from Eqs. tdi1/tdi2: chain A of
    X visits spacecraft 1 3 1 2 1 2 1 3 1 and chain B 1 2 1 3 1 3 1 2 1, X = A - B; a term's delay
    adds L_ij for each hop i -> j before it; summed: every L at t; nested: each L at the time the
    hop ends, t - (the delay so far).  Y, Z by the cyclic map.  (A ramp would not do for TDI-2: its
    summed X2 vanishes identically.)"""
    L0 = np.array([8.10, 8.25, 8.40, 8.20, 8.35, 8.05])
    rate = np.array([2e-6, -3e-6, 1e-6, -1e-6, 4e-6, -2e-6])  # s per s: nested - summed ~ 1e-4 s
    tk = synth.knot_grid(-2e6, 2e6, 1e5)
    pos = np.repeat(synth.static_triangle(np.zeros(1))[:, :, :1], len(tk), axis=2)
    delays = L0[:, None] + rate[:, None] * tk[None, :]
    o = oracle.Orbit(tk, pos, delays)
    N = 400
    t = synth.sample_grid(T0, DT, N)
    ys = lambda tt: (tt / 100.0) ** 2  # noqa: E731
    y = np.repeat(ys(t)[None, :], 6, axis=0)
    dm = oracle.DELAY_SUM if mode == "summed" else oracle.DELAY_NESTED
    xyz = oracle.tdi(P, gen, DT, T0, N, o, y, dm)
    Lf = lambda name, tt: L0[LINK_INDEX[name]] + rate[LINK_INDEX[name]] * tt  # noqa: E731
    seqs = ([1, 3, 1, 2, 1, 2, 1, 3, 1], [1, 2, 1, 3, 1, 3, 1, 2, 1])
    nterm = 4 if gen == 1 else 8
    ref = np.zeros((3, N))
    mag = np.zeros(N)
    for ch in range(3):
        cyc = lambda s: (s - 1 + ch) % 3 + 1  # noqa: E731
        for c, sign in ((0, 1.0), (1, -1.0)):
            seq = [cyc(s) for s in seqs[c]]
            D = np.zeros(N)
            ref[ch] += sign * ys(t)
            mag += ys(t)
            for q in range(1, nterm):
                hop = f"{seq[q - 1]}{seq[q]}"
                D = D + Lf(hop, t if mode == "summed" else t - D)
                ref[ch] += sign * ys(t - D)
                mag += ys(t - D)
    sl = slice(60, N - 30)  # away from the zero-extended ends
    tol = 1e-12 * mag[sl].max()
    assert np.abs(xyz[:, sl] - ref[:, sl]).max() <= tol
    if mode == "nested":  # the two forms really differ here
        summed = oracle.tdi(P, gen, DT, T0, N, o, y, oracle.DELAY_SUM)
        assert np.abs(summed[:, sl] - xyz[:, sl]).max() > 100 * tol
