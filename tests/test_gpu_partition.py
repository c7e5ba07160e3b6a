"""The multi-GPU splits run on one GPU (each rank's share one after the other) through the C ABI,
against the unsplit library run:
  - sources dealt by lr_partition_sources: every source's X, Y, Z equal bit for bit;
  - one long source split in time by lr_partition_time (halos from lr_valid_range, units of the
    plan's tile): the owned outputs equal bit for bit, in both precisions, and the ranks' adjoint
    partials (g on owned outputs only) add up to the unsplit sky-angle and strain gradients."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, dev, host  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
@pytest.mark.parametrize("ranks", [2, 3])
def test_time_split_matches_unsplit(ctx, precision, ranks):
    n, p = 200000, 25
    orb = synth.orbit_flexing(T0 - 3e5, T0 + n * DT + 3e5)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    src = synth.draw_sources(1, seed=31, A=1e-21)[0]
    s = (src.lam, src.beta, src.psi)
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    margin = synth.input_margin_samples(DT, p)
    full = lr.Plan(ctx, p, n, DT, o, t0=T0, precision=precision)
    ref = host(full.response(dev(hp), dev(hc), t0h, s))
    first, last = full.valid_range()
    hl, hr, tile = first, n - 1 - last, full.tile
    got = np.full_like(ref, np.nan)
    for r in range(ranks):
        sh = lr.partition_time(n, hl, hr, tile, ranks, r)
        m = sh.hi - sh.lo
        plan = lr.Plan(ctx, p, m, DT, o, t0=T0 + sh.lo * DT, precision=precision)
        win = slice(sh.lo, sh.hi + 2 * margin)
        x = host(plan.response(dev(hp[win]), dev(hc[win]), t0h + sh.lo * DT, s))
        plan.check()
        got[:, sh.first:sh.first + sh.count] = x[:, sh.first - sh.lo:sh.first - sh.lo + sh.count]
    np.testing.assert_array_equal(got, ref)


def test_time_split_adjoint_partials_add_up(ctx):
    n, p, ranks = 30000, 11, 3
    orb = synth.orbit_flexing(T0 - 3e5, T0 + n * DT + 3e5)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
    src = synth.draw_sources(1, seed=32, A=1e-21)[0]
    s = (src.lam, src.beta, src.psi)
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    margin = synth.input_margin_samples(DT, p)
    g = np.random.default_rng(4).standard_normal((3, n))
    full = lr.Plan(ctx, p, n, DT, o, t0=T0)
    ghp, ghc, gsky = (host(v) for v in full.backward(dev(hp), dev(hc), t0h, s, dev(g)))
    first, last = full.valid_range()
    acc_h = np.zeros((2, len(hp)))
    acc_s = np.zeros(3)
    for r in range(ranks):
        sh = lr.partition_time(n, first, n - 1 - last, full.tile, ranks, r)
        m = sh.hi - sh.lo
        plan = lr.Plan(ctx, p, m, DT, o, t0=T0 + sh.lo * DT)
        win = slice(sh.lo, sh.hi + 2 * margin)
        gs = np.zeros((3, m))
        own = slice(sh.first - sh.lo, sh.first - sh.lo + sh.count)
        gs[:, own] = g[:, sh.first:sh.first + sh.count]
        a, b, c = plan.backward(dev(hp[win]), dev(hc[win]), t0h + sh.lo * DT, s, dev(gs))
        plan.check()
        acc_h[0, win] += host(a)
        acc_h[1, win] += host(b)
        acc_s += host(c)
    gh = np.stack([ghp, ghc])
    assert np.linalg.norm(acc_h - gh) <= 1e-14 * np.linalg.norm(gh)
    oo = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    _, _, _, scale = oracle.backward(p, 2, DT, T0, n, oo, oo, hp, hc, t0h, *s, g, with_scale=True)
    assert np.all(np.abs(acc_s - gsky) <= np.maximum(1e-13 * np.abs(gsky), 4 * (p + 17) * 2.0 ** -53 * scale))


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_source_deal_matches_unsplit_batch(ctx, precision):
    import bench

    p, ranks = 25, 3
    lens, srcs = bench.workload(0, 1, 40)
    lens = (lens // 16).astype(np.int64)   # a short ragged batch
    h_off, out_off, t0h, sky, hp, hc = bench.build_inputs(lens, srcs, p)
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * int(lens.max()) + 3e5)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    plan = lr.Plan(ctx, p, 1, DT, o, t0=T0, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    ref = host(plan.response_batched(d(h_off), d(out_off), d(t0h), d(sky), d(hp), d(hc)))
    rank_of, _ = lr.partition_sources(lens, ranks)
    for r in range(ranks):
        sel = np.flatnonzero(rank_of == r)
        sub = bench.build_inputs(lens[sel], [srcs[i] for i in sel], p)
        x = host(plan.response_batched(*(d(a) for a in sub)))
        so = sub[1]
        for j, i in enumerate(sel):
            np.testing.assert_array_equal(x[3 * so[j]:3 * so[j + 1]], ref[3 * out_off[i]:3 * out_off[i + 1]])
    plan.check()
