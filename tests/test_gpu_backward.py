"""GPU parity of the adjoint (backward): transposes of the TDI and projection operators and
the sky-angle gradient, against the FP64 oracle and against finite differences."""
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


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def flex(ctx):
    return Pair(ctx, synth.orbit_flexing(-2e6, 4e6 * DT + 2e6))


def setup(ctx, orb, N, p, seed=1, precision=lr.FP64, gen=2):
    src = synth.draw_sources(1, seed=seed, A=1e-21)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, orb.gpu, t0=T0, precision=precision, generation=gen)
    return src, t0h, hp, hc, plan


@pytest.mark.parametrize("p", [5, 25])
def test_adjoint_identity_on_gpu(ctx, flex, p):
    """<R h, g> = <h, R^T g> with the library's own forward and backward (FP64)."""
    N = 20011
    src, t0h, hp, hc, plan = setup(ctx, flex, N, p)
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=len(hp)), rng.normal(size=len(hp))
    g = rng.normal(size=(3, N))
    Rh = host(plan.response(dev(a), dev(b), t0h, sky(src)))
    ghp, ghc, _ = plan.backward(dev(a), dev(b), t0h, sky(src), dev(g))
    plan.check()
    lhs = np.sum(Rh * g)
    rhs = np.sum(a * host(ghp)) + np.sum(b * host(ghc))
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(Rh * Rh) * np.sum(g * g))


@pytest.mark.parametrize("p,N", [(11, 6000), (25, 3001)])
def test_backward_matches_oracle(ctx, flex, p, N):
    src, t0h, hp, hc, plan = setup(ctx, flex, N, p, seed=2)
    rng = np.random.default_rng(4)
    g = rng.normal(size=(3, N))
    ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
    plan.check()
    rp, rc, rs, scale = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta,
                                        src.psi, g, with_scale=True)
    for got, ref in ((host(ghp), rp), (host(ghc), rc)):
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert_sky_close(host(gsky), rs, scale, p + 1)


def assert_sky_close(got, ref, scale, T):
    """1e-11 relative, or the rounding-error scale of the gradient sum, 4 (T + 16) u times the
    sum with every factor by its absolute value, when that is larger: at low frequency TDI
    cancels the strain by 1e4-1e6 and the sum of derivative reads against g_y cancels further,
    and the FP64 oracle's own sky gradient is then further than 1e-11 from the exact (binary128)
    value of its algorithm, while within that scale (tests/test_oracle_precision.py)."""
    K = 4 * (T + 16)
    bound = np.maximum(1e-11 * np.abs(ref), K * 2.0 ** -53 * scale)
    assert np.all(np.abs(got - ref) <= bound), (got, ref, bound)


def test_backward_first_generation_and_nested(ctx, flex):
    N, p = 4000, 11
    for gen, dm in ((1, lr.DELAY_SUM), (2, lr.DELAY_NESTED)):
        src = synth.draw_sources(1, seed=5, A=1e-21)[0]
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, generation=gen, delay_mode=dm)
        g = np.random.default_rng(6).normal(size=(3, N))
        ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src), dev(g))
        plan.check()
        rp, rc, rs, scale = oracle.backward(p, gen, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam,
                                            src.beta, src.psi, g, delay_mode=dm, with_scale=True)
        assert np.linalg.norm(host(ghp) - rp) <= 1e-11 * np.linalg.norm(rp)
        assert_sky_close(host(gsky), rs, scale, p + 1)


def loss_and_grad(plan, src, t0h, hp, hc, data, sigma, th=None):
    s = sky(src) if th is None else tuple(th)
    r = plan.response(dev(hp), dev(hc), t0h, s) - dev(data)
    return r, r / sigma ** 2


@pytest.mark.parametrize("N", [65536, synth.ONE_YEAR_SAMPLES])
def test_config4_gradients_by_central_differences(ctx, N):
    """Config-1 source plus white noise (sigma 1e-21, seed-fixed) on a static triangle; loss
    1/2 sum (R(h) - d)^2 / sigma^2.  Sky-angle gradients against central differences with
    step 1e-6 relative; strain gradients along random directions (exact for a quadratic)."""
    p, sigma = 25, 1e-21
    src = synth.config1_source()
    orb = Pair(ctx, synth.orbit_static(-2e6, N * DT + 2e6))
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, orb.gpu, t0=T0)
    clean = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
    data = clean + synth.white_noise(clean.shape, sigma)
    # evaluate at a slightly offset source so the residual carries signal as well as noise
    src2 = synth.Source(**{**src.__dict__, "lam": src.lam + 2e-3, "beta": src.beta - 1e-3, "psi": src.psi + 3e-3})
    r, g = loss_and_grad(plan, src2, t0h, hp, hc, data, sigma)
    ghp, ghc, gsky = plan.backward(dev(hp), dev(hc), t0h, sky(src2), g)
    plan.check()
    gsky = host(gsky)
    th0 = np.array([src2.lam, src2.beta, src2.psi])
    for i in range(3):
        e = 1e-6 * abs(th0[i])
        tp, tm = th0.copy(), th0.copy()
        tp[i] += e
        tm[i] -= e
        rp = plan.response(dev(hp), dev(hc), t0h, tuple(tp)) - dev(data)
        rm = plan.response(dev(hp), dev(hc), t0h, tuple(tm)) - dev(data)
        # L+ - L- = 1/2 sum (r+ - r-)(r+ + r-) / sigma^2, formed without cancellation
        fd = float(0.5 * torch.sum((rp - rm) * (rp + rm)).item() / sigma ** 2 / (2 * e))
        assert abs(fd - gsky[i]) <= 1e-6 * abs(gsky[i]), (i, fd, gsky[i])
    rng = np.random.default_rng(8)
    for _ in range(2):
        va, vb = rng.normal(size=len(hp)) * 1e-22, rng.normal(size=len(hp)) * 1e-22
        rp = plan.response(dev(hp + va), dev(hc + vb), t0h, sky(src2)) - dev(data)
        rm = plan.response(dev(hp - va), dev(hc - vb), t0h, sky(src2)) - dev(data)
        fd = float(0.5 * torch.sum((rp - rm) * (rp + rm)).item() / sigma ** 2 / 2.0)
        an = float(np.sum(host(ghp) * va) + np.sum(host(ghc) * vb))
        assert abs(fd - an) <= 1e-8 * abs(an)


def test_autograd_function(ctx, flex):
    N, p = 5000, 11
    src, t0h, hp, hc, plan = setup(ctx, flex, N, p, seed=9)
    a = dev(hp).requires_grad_(True)
    b = dev(hc).requires_grad_(True)
    s = torch.tensor([src.lam, src.beta, src.psi], dtype=torch.float64, device="cuda:0", requires_grad=True)
    xyz = lr.response(plan, a, b, s, t0h)
    w = torch.tensor(np.random.default_rng(1).normal(size=(3, N)), device="cuda:0")
    (xyz * w).sum().backward()
    rp, rc, rs, scale = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta,
                                        src.psi, host(w), with_scale=True)
    assert np.linalg.norm(host(a.grad) - rp) <= 1e-12 * np.linalg.norm(rp)
    assert_sky_close(host(s.grad), rs, scale, p + 1)


def test_batched_backward_matches_single(ctx, flex):
    p = 11
    lens = np.array([3000, 1, 0, 4500])
    srcs = synth.draw_sources(len(lens), seed=10, A=1e-21)
    m = synth.input_margin_samples(DT, p)
    h_off = np.concatenate([[0], np.cumsum(lens + 2 * m)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp = np.zeros(h_off[-1])
    hc = np.zeros(h_off[-1])
    t0h = np.full(len(lens), T0 - m * DT)
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, synth.sample_grid(t0h[s], DT, int(lens[s] + 2 * m)))
        hp[h_off[s]:h_off[s + 1]] = a
        hc[h_off[s]:h_off[s + 1]] = b
    skyarr = np.array([[s.lam, s.beta, s.psi] for s in srcs])
    g = np.random.default_rng(11).normal(size=3 * out_off[-1])
    plan = lr.Plan(ctx, p, 1, DT, flex.gpu, t0=T0)
    ghp, ghc, gsky = plan.backward_batched(torch.tensor(h_off, device="cuda:0"),
                                           torch.tensor(out_off, device="cuda:0"), dev(t0h), dev(skyarr),
                                           dev(hp), dev(hc), dev(g))
    plan.check()
    ghp, ghc, gsky = host(ghp), host(ghc), host(gsky)
    for s, src in enumerate(srcs):
        N = int(lens[s])
        sl = slice(h_off[s], h_off[s + 1])
        if N == 0:
            assert not np.any(ghp[sl]) and not np.any(gsky[s])
            continue
        gs = g[3 * out_off[s]:3 * out_off[s + 1]].reshape(3, N)
        rp, rc, rs, scale = oracle.backward(p, 2, DT, T0, N, flex.orc, flex.orc, hp[sl], hc[sl], t0h[s], src.lam,
                                            src.beta, src.psi, gs, with_scale=True)
        assert np.linalg.norm(ghp[sl] - rp) <= 1e-12 * np.linalg.norm(rp)
        assert np.linalg.norm(ghc[sl] - rc) <= 1e-12 * np.linalg.norm(rc)
        assert_sky_close(gsky[s], rs, scale, p + 1)
