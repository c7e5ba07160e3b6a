"""The mixed-precision adjoint (plans of precision LR_MIXED): TDI and projection transposes with
float-float weights and float-float accumulation on the FP32 pipe, FP64 positions and delays; the
sky gradient from float-float strain reads and derivative reads with FP64 geometry and assembly on
that g_y.  Against the FP64 oracle with white cotangents (residuals against noisy data, the
likelihood's use): strain gradients within 1e-6 relative L2; sky-angle gradients within 1e-6 or the
rounding scale of the gradient sum at FP32 precision, 4 (T + 16) u32 sum|terms| (the sum's terms
are up to ~1e8 times its value at low frequency); the adjoint identity against the mixed forward;
batched against single calls; central differences of the config-4 loss; the error for a smooth
cotangent (a noise-free residual) is reported."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, Pair, dev, host, sky  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def flex(ctx):
    return Pair(ctx, synth.orbit_flexing(-2e6, 4e6 * DT + 2e6))


def assert_sky_mixed(got, ref, scale, T):
    bound = np.maximum(1e-6 * np.abs(ref), 4 * (T + 16) * U32 * scale)
    assert np.all(np.abs(got - ref) <= bound), (got, ref, bound)


@pytest.mark.parametrize("p,N", [(11, 6000), (25, 4001), (41, 3000)])
@pytest.mark.parametrize("f", [1e-4, 3e-3])
def test_mixed_backward_against_oracle(ctx, flex, p, N, f):
    import dataclasses
    src = dataclasses.replace(synth.draw_sources(1, seed=2, A=1e-21)[0], f=f)
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=lr.MIXED)
    g = np.random.default_rng(4).normal(size=(3, N))
    ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
    plan.check()
    rp, rc, rs, scale = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta,
                                        src.psi, g, with_scale=True)
    eh = np.linalg.norm(np.r_[host(ghp) - rp, host(ghc) - rc]) / np.linalg.norm(np.r_[rp, rc])
    assert eh <= 1e-6, eh
    assert_sky_mixed(host(gsky), rs, scale, p + 1)


@pytest.mark.parametrize("p", [1, 3, 5, 7, 9, 13, 15, 17, 19, 21, 23, 31])
def test_mixed_backward_every_order(ctx, flex, p):
    """Every other compiled order of the mixed adjoint against the oracle: the TDI transpose's
    reference weights use per-order constant tables (order 1 has no far nodes at all, order 3
    two), and the gathers' tap windows change with the order."""
    import dataclasses
    N = 2500
    src = dataclasses.replace(synth.draw_sources(1, seed=6, A=1e-21)[0], f=3e-3)
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=lr.MIXED)
    g = np.random.default_rng(7).normal(size=(3, N))
    ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
    plan.check()
    rp, rc, rs, scale = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta,
                                        src.psi, g, with_scale=True)
    eh = np.linalg.norm(np.r_[host(ghp) - rp, host(ghc) - rc]) / np.linalg.norm(np.r_[rp, rc])
    assert eh <= 1e-6, eh
    assert_sky_mixed(host(gsky), rs, scale, p + 1)


def test_mixed_backward_nested_and_first_generation(ctx, flex):
    N, p = 4000, 11
    for gen, dm in ((1, lr.DELAY_SUM), (2, lr.DELAY_NESTED)):
        src = synth.draw_sources(1, seed=5, A=1e-21)[0]
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, generation=gen, delay_mode=dm, precision=lr.MIXED)
        g = np.random.default_rng(6).normal(size=(3, N))
        ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
        plan.check()
        rp, rc, rs, scale = oracle.backward(p, gen, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam,
                                            src.beta, src.psi, g, delay_mode=dm, with_scale=True)
        assert np.linalg.norm(host(ghp) - rp) <= 1e-6 * np.linalg.norm(rp)
        assert_sky_mixed(host(gsky), rs, scale, p + 1)


@pytest.mark.parametrize("p", [11, 25])
def test_mixed_adjoint_identity(ctx, flex, p):
    """<R h, g> = <h, R^T g> with the mixed forward and the mixed adjoint, to their accuracy."""
    N = 20011
    src = synth.draw_sources(1, seed=1, A=1e-21)[0]
    t0h, _, _ = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=lr.MIXED)
    rng = np.random.default_rng(3)
    m = synth.input_margin_samples(DT, p)
    a, b = rng.normal(size=N + 2 * m), rng.normal(size=N + 2 * m)
    g = rng.normal(size=(3, N))
    Rh = host(plan.response(dev(a), dev(b), t0h, sky(src)))
    ghp, ghc, _ = plan.backward(dev(a), dev(b), t0h, sky(src), dev(g))
    plan.check()
    lhs = np.sum(Rh * g)
    rhs = np.sum(a * host(ghp)) + np.sum(b * host(ghc))
    assert abs(lhs - rhs) <= 1e-6 * np.sqrt(np.sum(Rh * Rh) * np.sum(g * g))


def test_mixed_batched_backward_matches_single(ctx, flex):
    p = 11
    lens = np.array([3000, 1, 0, 4500])
    srcs = synth.draw_sources(len(lens), seed=10, A=1e-21)
    m = synth.input_margin_samples(DT, p)
    h_off = np.concatenate([[0], np.cumsum(lens + 2 * m)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp, hc = np.zeros(h_off[-1]), np.zeros(h_off[-1])
    t0h = np.full(len(lens), T0 - m * DT)
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, synth.sample_grid(t0h[s], DT, int(lens[s] + 2 * m)))
        hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]] = a, b
    skyarr = np.array([[s.lam, s.beta, s.psi] for s in srcs])
    g = np.random.default_rng(11).normal(size=3 * out_off[-1])
    plan = lr.Plan(ctx, p, 1, DT, flex.gpu, t0=T0, precision=lr.MIXED)
    ghp, ghc, gsky = plan.backward_batched(torch.tensor(h_off, device="cuda:0"), torch.tensor(out_off, device="cuda:0"),
                                           dev(t0h), dev(skyarr), dev(hp), dev(hc), dev(g))
    plan.check()
    ghp, ghc, gsky = host(ghp), host(ghc), host(gsky)
    for s, src in enumerate(srcs):
        N = int(lens[s])
        sl = slice(h_off[s], h_off[s + 1])
        if N == 0:
            assert not np.any(ghp[sl]) and not np.any(gsky[s])
            continue
        single = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=lr.MIXED)
        gs = g[3 * out_off[s]:3 * out_off[s + 1]]
        a, b, c = (host(v) for v in single.backward(dev(hp[sl]), dev(hc[sl]), t0h[s], tuple(skyarr[s]), dev(gs)))
        single.check()
        np.testing.assert_allclose(ghp[sl], a, rtol=0, atol=1e-14 * max(np.abs(a).max(), 1e-300))
        np.testing.assert_allclose(ghc[sl], b, rtol=0, atol=1e-14 * max(np.abs(b).max(), 1e-300))
        np.testing.assert_allclose(gsky[s], c, rtol=1e-12)


def test_config4_mixed_gradients_by_central_differences(ctx):
    """Config 4 (config-1 source, static triangle, white noise sigma 1e-21, N = 65 536): the mixed
    plan's gradients of the loss against central differences of the loss itself, evaluated by the
    FP64 plan (a difference quotient of the mixed forward would carry its ~1e-8 rounding divided
    by the step): strain gradients along random directions, sky angles with step 1e-6 relative,
    agreement 1e-6."""
    N, p, sigma = 65536, 25, 1e-21
    src = synth.config1_source()
    orb = Pair(ctx, synth.orbit_static(-2e6, N * DT + 2e6))
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    mixed = lr.Plan(ctx, p, N, DT, orb.gpu, t0=T0, precision=lr.MIXED)
    plan = lr.Plan(ctx, p, N, DT, orb.gpu, t0=T0)  # the loss
    clean = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
    data = clean + synth.white_noise(clean.shape, sigma)
    src2 = synth.Source(**{**src.__dict__, "lam": src.lam + 2e-3, "beta": src.beta - 1e-3, "psi": src.psi + 3e-3})
    r = plan.response(dev(hp), dev(hc), t0h, sky(src2)) - dev(data)
    g = r / sigma ** 2
    ghp, ghc, gsky = mixed.backward(dev(hp), dev(hc), t0h, sky(src2), g)
    mixed.check()
    gsky = host(gsky)
    th0 = np.array([src2.lam, src2.beta, src2.psi])
    for i in range(3):
        e = 1e-6 * abs(th0[i])
        tp, tm = th0.copy(), th0.copy()
        tp[i] += e
        tm[i] -= e
        rp = plan.response(dev(hp), dev(hc), t0h, tuple(tp)) - dev(data)
        rm = plan.response(dev(hp), dev(hc), t0h, tuple(tm)) - dev(data)
        fd = float(0.5 * torch.sum((rp - rm) * (rp + rm)).item() / sigma ** 2 / (2 * e))
        assert abs(fd - gsky[i]) <= 1e-6 * abs(gsky[i]), (i, fd, gsky[i])
    rng = np.random.default_rng(8)
    for _ in range(2):
        va, vb = rng.normal(size=len(hp)) * 1e-22, rng.normal(size=len(hp)) * 1e-22
        rp = plan.response(dev(hp + va), dev(hc + vb), t0h, sky(src2)) - dev(data)
        rm = plan.response(dev(hp - va), dev(hc - vb), t0h, sky(src2)) - dev(data)
        fd = float(0.5 * torch.sum((rp - rm) * (rp + rm)).item() / sigma ** 2 / 2.0)
        an = float(np.sum(host(ghp) * va) + np.sum(host(ghc) * vb))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_smooth_cotangent_is_reported(ctx, flex, capsys):
    """A noise-free residual (as smooth as the signal) cancels in the transposed operators as the
    signal does in the forward ones: the mixed adjoint's error for it is reported."""
    import dataclasses
    N, p = 4001, 25
    out = []
    for f in (1e-4, 1e-3, 1e-2):
        src = dataclasses.replace(synth.draw_sources(1, seed=2, A=1e-21)[0], f=f)
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        g = oracle.response(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta, src.psi) * 1e21
        plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=lr.MIXED)
        ghp, ghc, _ = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
        plan.check()
        rp, rc, _ = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta, src.psi, g)
        eh = np.linalg.norm(np.r_[host(ghp) - rp, host(ghc) - rc]) / np.linalg.norm(np.r_[rp, rc])
        assert np.isfinite(eh)
        out.append((f, eh))
    with capsys.disabled():
        print("\nmixed adjoint, smooth cotangent: " + ", ".join(f"f={f:.0e}: rel L2 {e:.2e}" for f, e in out))
