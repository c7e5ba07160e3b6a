"""Pins the oracle's windowed evaluator (oracle.response_at: y recomputed over a local window
around each requested output, then TDI read from that window) to the full-series oracle
(oracle.response: y over the whole output span, then TDI; Eqs. instrument-response-to-gw,
tdi1, tdi2).  Every long-series parity check samples outputs through response_at, so a window
one sample short, a maximum delay taken in the wrong delay mode or a wrong zero-extension edge
must show up here.  Both evaluate the same reads with the same integer base and fractional
offset, so the results must agree bit for bit."""
import numpy as np
import pytest

import oracle
import synth

DT, T0 = 10.0, 0.0
N = 1500


@pytest.fixture(scope="module")
def flexing():
    orb = synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5)
    return oracle.Orbit(orb.t_knots, orb.pos, None)


def _indices(n, tile=340, seed=0):
    rng = np.random.default_rng(seed)
    edges = [0, 1, 2, 3, n - 3, n - 2, n - 1]
    for t in range(tile, n, tile):
        edges += [t - 1, t, t + 1]
    return np.unique(np.concatenate([edges, rng.integers(0, n, 40)]).astype(np.int64))


@pytest.mark.parametrize("p", [1, 11, 25, 41])
@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("mode", [oracle.DELAY_SUM, oracle.DELAY_NESTED])
def test_windowed_matches_full(flexing, p, gen, mode):
    src = synth.draw_sources(1, seed=100 + p + gen)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    args = (p, gen, DT, T0, N, flexing, flexing, hp, hc, t0h, src.lam, src.beta, src.psi)
    idx = _indices(N)
    full = oracle.response(*args, delay_mode=mode)
    win = oracle.response_at(*args, idx, delay_mode=mode)
    np.testing.assert_array_equal(win, full[:, idx])
    # the rounding-error scale used by the tolerances takes the same path
    full_abs = oracle.response(*args, delay_mode=mode, absval=True)
    win_abs = oracle.response_at(*args, idx, delay_mode=mode, absval=True)
    np.testing.assert_array_equal(win_abs, full_abs[:, idx])


def test_windowed_hybrid_orbits():
    """Projection and TDI orbits differ (the hybrid template): the window must follow the TDI
    orbit's delays, and the link series the projection orbit's geometry."""
    porb = synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5)
    torb = synth.orbit_equal_arm(T0 - 3e5, T0 + N * DT + 3e5)
    po = oracle.Orbit(porb.t_knots, porb.pos, None)
    to = oracle.Orbit(torb.t_knots, torb.pos, None)
    src = synth.draw_sources(1, seed=7)[0]
    p = 25
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    args = (p, 2, DT, T0, N, po, to, hp, hc, t0h, src.lam, src.beta, src.psi)
    idx = _indices(N, seed=3)
    np.testing.assert_array_equal(oracle.response_at(*args, idx), oracle.response(*args)[:, idx])


def test_windowed_short_series_edges(flexing):
    """A series shorter than the TDI reach: every output's window runs past both ends, where
    the link series are zero."""
    n = 40
    src = synth.draw_sources(1, seed=9)[0]
    p = 25
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    args = (p, 2, DT, T0, n, flexing, flexing, hp, hc, t0h, src.lam, src.beta, src.psi)
    idx = np.arange(n, dtype=np.int64)
    np.testing.assert_array_equal(oracle.response_at(*args, idx), oracle.response(*args))
