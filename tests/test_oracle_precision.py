"""How far the FP64 oracle is from the exact result of its own algorithm.

The reference values come from the oracle's own source compiled with every `double` widened to
IEEE binary128 (oracle/lr_oracle_quad.c: same steps, same order, same constants; rounding ~2^-113
instead of 2^-53), so |oracle64 - oracle128| is the FP64 oracle's own rounding error.

This is the evidence behind the FP64 parity tolerances of the GPU tests:
  - at low frequency the response is a difference of nearly equal reads (|y|/|h| ~ 2 pi f L) that
    TDI-2 cancels again, so a plain FP64 evaluation of the definition is itself further than 1e-12
    from the exact value (here 0.1 mHz: ~5e-12), while at 3 mHz and above it is within 1e-12;
  - the rounding-error scale K u ||E|| (K = 2 (T + 16), E = the response with |weights|,
    |coefficients| and |inputs|) bounds that error everywhere;
  - the same holds for the sky-angle gradient with 4 (T + 16) u times its absolute-value scale: the
    FP64 oracle misses 1e-11 there by an order of magnitude at 0.1 mHz, while the strain gradient
    stays near 1e-14.
"""
import dataclasses
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

DT, T0 = 10.0, 0.0
U64 = 2.0 ** -53

pytestmark = pytest.mark.skipif(not oracle.quad_available(), reason="no binary128 libm in this toolchain")


def test_quad_build_uses_binary128_math():
    """Every libm call of the widened oracle goes to its binary128 version (a call left at FP64
    would cap the reference at FP64 accuracy)."""
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    oracle.build()
    out = subprocess.run(["nm", "-D", "--undefined-only", oracle._LIB_Q], capture_output=True, text=True,
                         check=True).stdout
    names = {line.split()[-1].split("@")[0] for line in out.splitlines() if line.strip()}
    assert {"sqrtf128", "sinf128", "cosf128", "floorf128"} <= names
    assert not names & {"sqrt", "sin", "cos", "floor", "ceil", "fabs"}


@pytest.fixture(scope="module")
def flexing():
    n = 2000
    orb = synth.orbit_flexing(T0 - 3e5, T0 + n * DT + 3e5)
    return n, orb, oracle.Orbit(orb.t_knots, orb.pos, orb.delays)


def _case(n, p, orb, o, f, seed=11):
    src = dataclasses.replace(synth.draw_sources(1, seed=seed)[0], f=f)
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    args = (p, 2, DT, T0, n, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    exact = oracle.response_quad(p, 2, DT, T0, n, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h,
                                 src.lam, src.beta, src.psi)
    return args, exact


@pytest.mark.parametrize("f", [1e-4, 3e-4, 1e-3, 3e-3, 1e-2])
def test_fp64_response_error_against_binary128(flexing, f):
    n, orb, o = flexing
    p = 25
    args, exact = _case(n, p, orb, o, f)
    r64 = oracle.response(*args)
    scale = oracle.response(*args, absval=True)
    err = np.linalg.norm(r64 - exact)
    rel = err / np.linalg.norm(exact)
    # the rounding-error scale bounds the FP64 oracle's own error at every frequency
    assert err <= 2 * (p + 17) * U64 * np.linalg.norm(scale)
    if f <= 1e-4:
        # and a plain FP64 evaluation of the definition is itself further than 1e-12 from the
        # exact value there: no FP64 program can be held to 1e-12 against it
        assert rel > 1e-12
    if f >= 3e-3:
        assert rel < 1e-12


def test_windowed_binary128_matches_full(flexing):
    """The sampled binary128 evaluator (used for long series) equals the full one bit for bit."""
    n, orb, o = flexing
    p = 11
    src = synth.draw_sources(1, seed=4)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    qa = (p, 2, DT, T0, n, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h, src.lam, src.beta, src.psi)
    idx = np.array([0, 1, 2, 339, 340, 1000, n - 2, n - 1], dtype=np.int64)
    np.testing.assert_array_equal(oracle.response_at_quad(*qa, idx), oracle.response_quad(*qa)[:, idx])


@pytest.mark.parametrize("f,kind", [(1e-4, "white"), (3e-4, "smooth"), (3e-3, "white")])
def test_fp64_gradient_error_against_binary128(f, kind):
    n, p = 300, 11
    orb = synth.orbit_flexing(T0 - 3e5, T0 + n * DT + 3e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    src = dataclasses.replace(synth.draw_sources(1, seed=11)[0], f=f)
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    args = (p, 2, DT, T0, n, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    if kind == "white":   # residuals against noisy data
        g = np.random.default_rng(5).standard_normal((3, n))
    else:                 # a noise-free residual: as smooth as the signal
        g = oracle.response(*args) * 1e21
    ghp, ghc, gsky, scale = oracle.backward(*args, g, with_scale=True)
    qhp, qhc, qsky = oracle.backward_quad(p, 2, DT, T0, n, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h,
                                          src.lam, src.beta, src.psi, g)
    eh = np.linalg.norm(np.r_[ghp - qhp, ghc - qhc]) / np.linalg.norm(np.r_[qhp, qhc])
    assert eh < 1e-12  # the strain gradient has no cancellation
    err = np.abs(gsky - qsky)
    assert np.all(err <= 4 * (p + 17) * U64 * scale)
    if f <= 1e-4:
        # the sky gradient of a plain FP64 evaluation is itself further than 1e-11 from exact
        assert np.max(err / np.abs(qsky)) > 1e-11
