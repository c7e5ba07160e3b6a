"""Galactic binaries generated on the device (Sec. "Template generation") through the C ABI:
  - lr_gb_polarisations against the oracle's formula evaluated in binary128 (the exact values):
    within a few units in the last place of the amplitude at one-year times;
  - lr_response_gb against the oracle's response to the exact polarisations (rounded once to FP64),
    both precisions, with the parity bounds of the strain-array path;
  - every source of the batched generated-strain calls against the same oracle, and the generated-
    template log-likelihood against the oracle's inner products of the X, Y, Z the call returns."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, Pair, assert_close, dev, host  # noqa: E402

if not oracle.quad_available():
    pytest.skip("no binary128 libm in this toolchain", allow_module_level=True)


def gb_of(src):
    return (src.A, src.f, src.fdot, src.fddot_value(), src.phi0, src.iota)


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.mark.parametrize("f", [1e-4, 1e-2])
def test_generator_against_binary128(ctx, f):
    src = synth.draw_sources(1, seed=80, A=1e-21, fdot=1e-16)[0]
    g = list(gb_of(src))
    g[1] = f
    g[3] = 11 * g[2] ** 2 / (3 * f)
    t0, n = 3.0e7, 4096
    hp, hc = lr.gb_polarisations(g, t0, DT, n)
    qp, qc = oracle.gb_polarisations(*g, t0, DT, n, quad=True)
    ci = np.cos(src.iota)
    amp = src.A * (1 + ci * ci)
    ulp = np.spacing(amp)
    assert np.max(np.abs(host(hp) - qp)) <= 8 * ulp
    assert np.max(np.abs(host(hc) - qc)) <= 8 * ulp


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
@pytest.mark.parametrize("f", [1e-4, 3e-3, 1e-2])
def test_response_gb_against_oracle(ctx, precision, rel, f):
    N, p, t0 = 20000, 25, 1.0e7
    pair = Pair(ctx, synth.orbit_flexing(t0 - 3e5, t0 + N * DT + 3e5))
    src = synth.draw_sources(1, seed=81, A=1e-21, fdot=1e-17)[0]
    g = list(gb_of(src))
    g[1] = f
    g[3] = 11 * g[2] ** 2 / (3 * f)
    sky = (src.lam, src.beta, src.psi)
    plan = lr.Plan(ctx, p, N, DT, pair.gpu, t0=t0, precision=precision)
    got = host(plan.response_gb(g, sky))
    plan.check()
    m = synth.input_margin_samples(DT, p)
    t0h = t0 - m * DT
    hp, hc = oracle.gb_polarisations(*g, t0h, DT, N + 2 * m, quad=True)
    args = (p, 2, DT, t0, N, pair.orc, pair.orc, hp, hc, t0h, *sky)
    ref = oracle.response(*args)
    scale = oracle.response(*args, absval=True)
    assert_close(got, ref, scale, p + 1, rel, f"generated strain f={f}")


def batch(lens, seed):
    srcs = synth.draw_sources(len(lens), seed=seed, A=1e-22, fdot=1e-17)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    gbs = np.array([gb_of(s) for s in srcs])
    sky = np.array([[s.lam, s.beta, s.psi] for s in srcs])
    return srcs, out_off, gbs, sky


def epilogue_bound(xyz, data, w, k):
    a = np.abs(oracle.aet(xyz))
    wa = np.asarray(w)[:, None]
    return k * float(np.sum(wa * a * np.abs(data))), k * float(np.sum(wa * a * a))


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_batched_generated_strain(ctx, precision, rel):
    """Every source of lr_response_gb_batched against the oracle fed with the exact polarisations;
    lr_log_likelihood_gb_batched's X, Y, Z equal the response's and its values equal the oracle's
    inner products of those X, Y, Z within the epilogue's rounding bound."""
    p, t0 = 25, 0.0
    lens = [3000, 0, 1, 20011, 341, 9000]
    srcs, out_off, gbs, sky = batch(lens, 82)
    pair = Pair(ctx, synth.orbit_flexing(t0 - 3e5, t0 + max(lens) * DT + 3e5))
    plan = lr.Plan(ctx, p, 1, DT, pair.gpu, t0=t0, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    got = host(plan.response_gb_batched(d(out_off), d(gbs), d(sky)))
    plan.check()
    m = synth.input_margin_samples(DT, p)
    for s, n in enumerate(lens):
        if n == 0:
            continue
        hp, hc = oracle.gb_polarisations(*gbs[s], t0 - m * DT, DT, n + 2 * m, quad=True)
        args = (p, 2, DT, t0, n, pair.orc, pair.orc, hp, hc, t0 - m * DT, *sky[s])
        ref = oracle.response(*args)
        scale = oracle.response(*args, absval=True)
        assert_close(got[3 * out_off[s]:3 * out_off[s + 1]].reshape(3, n), ref, scale, p + 1, rel, f"source {s}")
    data = np.random.default_rng(3).normal(size=3 * int(out_off[-1])) * 1e-21
    w = (1e42, 2e42, 0.5e42)
    xyz = torch.empty(3 * int(out_off[-1]), dtype=torch.float64, device="cuda:0")
    logl = host(plan.log_likelihood_gb_batched(d(out_off), d(gbs), d(sky), d(data), w, xyz=xyz))
    plan.check()
    xh = host(xyz)
    assert np.array_equal(xh, got)
    k = 1e-12 if precision == lr.FP64 else 4e-6
    for s, n in enumerate(lens):
        sl = slice(3 * out_off[s], 3 * out_off[s + 1])
        if n == 0:
            assert logl[s] == 0.0
            continue
        x, dd = xh[sl].reshape(3, n), data[sl].reshape(3, n)
        dh, hh = oracle.like_inner(x, dd, w)
        bdh, bhh = epilogue_bound(x, dd, w, k)
        assert abs(logl[s] - (dh - 0.5 * hh)) <= bdh + 0.5 * bhh + 4 * 2.0 ** -53 * (abs(dh) + abs(hh))
