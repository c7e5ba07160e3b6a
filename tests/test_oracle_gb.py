"""Pins the oracle's Galactic-binary polarisations (Sec. "Template generation") to the formula's
closed values and invariants: the value at the reference time, the amplitude identity
(h+/A+)^2 + (hx/Ax)^2 = 1, and the instantaneous frequency dPhi/dt / (2 pi) = f0 + fdot t +
fddot t^2 / 2 from central differences of the unwrapped phase (with exaggerated derivatives, so a
wrong factor on fdot or fddot fails).  The binary128 build of the same formula agrees with the FP64
one where FP64 is accurate and shows the FP64 phase rounding at one year and 10 mHz."""
import numpy as np
import pytest

import oracle

A, IOTA, PHI0 = 1e-22, 0.7, 1.3


def amps():
    ci = np.cos(IOTA)
    return A * (1 + ci * ci), 2 * A * ci


def test_value_at_reference_time():
    hp, hc = oracle.gb_polarisations(A, 3e-3, 1e-17, 0.0, PHI0, IOTA, 0.0, 10.0, 1)
    ap, ax = amps()
    assert hp[0] == pytest.approx(ap * np.cos(PHI0), rel=1e-15)
    assert hc[0] == pytest.approx(ax * np.sin(PHI0), rel=1e-15)


def test_amplitude_identity():
    hp, hc = oracle.gb_polarisations(A, 3e-3, 1e-17, 1e-30, PHI0, IOTA, 1e6, 10.0, 5000)
    ap, ax = amps()
    np.testing.assert_allclose((hp / ap) ** 2 + (hc / ax) ** 2, 1.0, rtol=0, atol=1e-14)


def test_instantaneous_frequency():
    f0, fd, fdd = 1e-3, 2e-9, 3e-14
    dt, t0, n = 1.0, 0.0, 20001
    hp, hc = oracle.gb_polarisations(A, f0, fd, fdd, PHI0, IOTA, t0, dt, n)
    ap, ax = amps()
    ph = np.unwrap(np.arctan2(hc / ax, hp / ap))
    t = t0 + dt * np.arange(n)
    f_num = (ph[2:] - ph[:-2]) / (2 * dt) / (2 * np.pi)
    f_true = f0 + fd * t[1:-1] + 0.5 * fdd * t[1:-1] ** 2
    # central differences of a cubic phase: error 2 pi fdd dt^2 / 6 / (2 pi), plus phase rounding
    np.testing.assert_allclose(f_num, f_true, rtol=0, atol=1e-11)


@pytest.mark.skipif(not oracle.quad_available(), reason="no binary128 libm in this toolchain")
def test_binary128_formula():
    args = (A, 1e-2, 1e-17, 11 * 1e-34 / 3e-2, PHI0, IOTA)
    ap, _ = amps()
    hp, _ = oracle.gb_polarisations(*args, 0.0, 10.0, 200)
    qp, _ = oracle.gb_polarisations(*args, 0.0, 10.0, 200, quad=True)
    assert np.max(np.abs(hp - qp)) <= 1e-13 * ap     # early times: FP64 is accurate
    hp, _ = oracle.gb_polarisations(*args, 3.0e7, 10.0, 200)
    qp, _ = oracle.gb_polarisations(*args, 3.0e7, 10.0, 200, quad=True)
    assert np.max(np.abs(hp - qp)) > 1e-12 * ap      # one year at 10 mHz: FP64 phase rounding shows
