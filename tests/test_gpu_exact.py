"""GPU parity against the exact result: the oracle's own source evaluated in binary128
(oracle.response_quad / response_at_quad / backward_quad), rounded once to FP64.

Against the exact value the FP64 build must be within 1e-12 where a plain FP64 evaluation of the
definition (the FP64 oracle) is, and otherwise no further from it than that FP64 evaluation
(with 25 % slack): at low frequency the response is ill-conditioned and no FP64 program reaches
1e-12 (tests/test_oracle_precision.py).  The mixed build must be within 1e-6.  Also checks
lr_valid_range: inside it the outputs do not depend on the output span's edges."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, dev, host, parity_bound  # noqa: E402

SLACK = 1.25

if not oracle.quad_available():
    pytest.skip("no binary128 libm in this toolchain", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    oracle.set_threads_quad(16)
    return lr.Context(0)


def fp64_bound(exact, r64):
    """max(1e-12 ||exact||, SLACK * ||oracle64 - exact||)"""
    return max(1e-12 * np.linalg.norm(exact), SLACK * np.linalg.norm(r64 - exact))


@pytest.mark.parametrize("p", [11, 25, 41])
@pytest.mark.parametrize("f", [1e-4, 1e-3, 1e-2])
def test_fused_response_against_binary128(ctx, p, f):
    N = 2500
    orb = synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    g = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
    src = dataclasses.replace(synth.draw_sources(1, seed=21)[0], f=f)
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    s = (src.lam, src.beta, src.psi)
    exact = oracle.response_quad(p, 2, DT, T0, N, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h, *s)
    r64 = oracle.response(p, 2, DT, T0, N, o, o, hp, hc, t0h, *s)
    for prec in (lr.FP64, lr.MIXED):
        plan = lr.Plan(ctx, p, N, DT, g, t0=T0, precision=prec)
        got = host(plan.response(dev(hp), dev(hc), t0h, s))
        plan.check()
        err = np.linalg.norm(got - exact)
        if prec == lr.FP64:
            assert err <= fp64_bound(exact, r64), (err / np.linalg.norm(exact), np.linalg.norm(r64 - exact))
        else:
            assert err <= 1e-6 * np.linalg.norm(exact)


def test_one_year_sampled_against_binary128(ctx):
    """One-year sources of the batch's frequency range, sampled outputs through the windowed
    binary128 evaluator, FP64 build."""
    N, p = synth.ONE_YEAR_SAMPLES, 25
    orb = synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    g = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
    plan = lr.Plan(ctx, p, N, DT, g, t0=T0, precision=lr.FP64)
    rng = np.random.default_rng(8)
    idx = np.sort(np.concatenate([[0, 1, N - 1], rng.integers(0, N, 40)])).astype(np.int64)
    for f in (1e-4, 2e-3):
        src = dataclasses.replace(synth.draw_sources(1, seed=22)[0], f=f)
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        s = (src.lam, src.beta, src.psi)
        got = host(plan.response(dev(hp), dev(hc), t0h, s))[:, idx]
        plan.check()
        exact = oracle.response_at_quad(p, 2, DT, T0, N, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h, *s, idx)
        r64 = oracle.response_at(p, 2, DT, T0, N, o, o, hp, hc, t0h, *s, idx)
        assert np.linalg.norm(got - exact) <= fp64_bound(exact, r64)


@pytest.mark.parametrize("f", [1e-4, 3e-3])
def test_sky_gradient_against_binary128(ctx, f):
    N, p = 600, 11
    orb = synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    g = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
    src = dataclasses.replace(synth.draw_sources(1, seed=23)[0], f=f)
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    s = (src.lam, src.beta, src.psi)
    gx = np.random.default_rng(9).standard_normal((3, N))
    plan = lr.Plan(ctx, p, N, DT, g, t0=T0)
    ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, s, dev(gx))
    plan.check()
    qhp, qhc, qsky = oracle.backward_quad(p, 2, DT, T0, N, orb.t_knots, orb.pos, orb.delays, hp, hc, t0h, *s, gx)
    _, _, rsky, scale = oracle.backward(p, 2, DT, T0, N, o, o, hp, hc, t0h, *s, gx, with_scale=True)
    gh = np.r_[host(ghp), host(ghc)]
    qh = np.r_[qhp, qhc]
    assert np.linalg.norm(gh - qh) <= 1e-12 * np.linalg.norm(qh)
    # The sky gradient is a sum whose terms are up to ~1e10 times its value at low frequency: any
    # FP64 summation order lands at a random point within u times the sum of |terms|, the FP64
    # oracle included (it is not a closer reference here), so the bound is that rounding scale,
    # 4 (T + 16) u scale, shown to bound a plain FP64 evaluation in tests/test_oracle_precision.py.
    bound = np.maximum(1e-11 * np.abs(qsky), 4 * (p + 17) * 2.0 ** -53 * scale)
    assert np.all(np.abs(host(gsky) - qsky) <= bound), (host(gsky) - qsky, rsky - qsky, bound)


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_valid_range_outputs_do_not_see_the_span_edges(ctx, precision, rel):
    """Outputs in lr_valid_range equal those of a longer span (the oracle on [-K, N + K)); the
    first output of the short span does not (it reads the zero extension)."""
    N, K, p = 3000, 400, 25
    orb = synth.orbit_flexing(T0 - 6e5, T0 + (N + K) * DT + 6e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    g = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    src = synth.draw_sources(1, seed=24, A=1e-21)[0]
    s = (src.lam, src.beta, src.psi)
    t0_long = T0 - K * DT
    t0h, hp, hc = synth.gb_input(src, t0_long, DT, N + 2 * K, p)
    plan = lr.Plan(ctx, p, N, DT, g, t0=T0, precision=precision)
    first, last = plan.valid_range()
    assert 0 < first < 200 and last == N - 2 - (p - 1) // 2
    got = host(plan.response(dev(hp), dev(hc), t0h, s))
    plan.check()
    largs = (p, 2, DT, t0_long, N + 2 * K, o, o, hp, hc, t0h, *s)
    ref = oracle.response(*largs)[:, K:K + N]
    scale = oracle.response(*largs, absval=True)[:, K:K + N]
    inside = slice(first, last + 1)
    err = np.linalg.norm(got[:, inside] - ref[:, inside])
    assert err <= parity_bound(ref[:, inside], scale[:, inside], p + 1, rel)
    assert np.linalg.norm(got[:, :1] - ref[:, :1]) > 1e-3 * np.linalg.norm(ref[:, :1])
