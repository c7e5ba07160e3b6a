"""GPU parity of the mixed-precision forward response (FP32 taps and accumulation of the
interpolated strain, float-float link series, FP64 times / splines / delays) against the FP64
oracle: relative L2 <= 1e-6 per source across the 0.1-10 mHz band."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, Pair, assert_close, dev, host, run_case, sky  # noqa: E402

RELMX = 1e-6


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def orbits(ctx):
    span = (-2e6, 6e5 * DT + 2e6)
    return {"flex": Pair(ctx, synth.orbit_flexing(*span)), "eq": Pair(ctx, synth.orbit_equal_arm(*span)),
            "static": Pair(ctx, synth.orbit_static(*span))}


def mixed(ctx, src, N, p, porb, torb=None, **kw):
    return run_case(ctx, src, N, p, porb, torb, precision=lr.MIXED, rel=RELMX, **kw)


def test_config1_mixed(ctx, orbits):
    src = synth.config1_source()
    for kind in ("project", "tdi", "response"):
        e = mixed(ctx, src, 65536, 25, orbits["static"], kind=kind)
        assert e < RELMX


@pytest.mark.parametrize("f", [1e-4, 3e-4, 1e-3, 3e-3, 1e-2])
def test_frequency_band_flexing(ctx, orbits, f):
    src = synth.Source(A=1e-21, f=f, fdot=1e-17, phi0=0.3, iota=0.7, psi=0.4, lam=1.0, beta=0.3)
    e = mixed(ctx, src, 30000, 25, orbits["flex"])
    assert e < RELMX


@pytest.mark.parametrize("p", [1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 31, 41])
def test_orders(ctx, orbits, p):
    src = synth.Source(A=1e-21, f=2e-3, fdot=1e-17, phi0=0.3, iota=0.7, psi=0.4, lam=1.0, beta=0.3)
    mixed(ctx, src, 12345, p, orbits["flex"])


@pytest.mark.parametrize("template", ["equal_arm", "hybrid"])
def test_templates(ctx, orbits, template):
    src = synth.draw_sources(1, seed=1, A=1e-21)[0]
    porb = orbits["eq"] if template == "equal_arm" else orbits["flex"]
    mixed(ctx, src, 40000, 25, porb, orbits["eq"])


@pytest.mark.parametrize("kind", ["project", "tdi"])
def test_unfused_stages(ctx, orbits, kind):
    src = synth.draw_sources(1, seed=2, A=1e-21)[0]
    mixed(ctx, src, 30011, 25, orbits["flex"], kind=kind)


def test_first_generation(ctx, orbits):
    src = synth.draw_sources(1, seed=3, A=1e-21)[0]
    mixed(ctx, src, 20000, 25, orbits["flex"], gen=1)


@pytest.mark.parametrize("N,tile", [(1, 0), (7, 0), (255, 256), (257, 256), (1000, 128), (1000, 18), (4096, 340)])
def test_small_and_ragged(ctx, orbits, N, tile):
    """Tiles that are not whole TDI items (18) and the largest tile the staged arrays hold (340)."""
    src = synth.draw_sources(1, seed=4, A=1e-21)[0]
    mixed(ctx, src, N, 25, orbits["flex"], tile=tile)


def test_sky_along_an_arm(ctx, orbits):
    """Sky direction 1.4e-3 rad from arm 12 at mid-span on the flexing orbit: 1/(2(1 - k.n)) and
    the patterns then change by a large fraction over one tile, which the tile's geometry cubic
    must carry at float-float accuracy."""
    N = 20000
    orb = orbits["flex"].orb
    tm = 0.5 * N * DT
    x = np.array([[np.interp(tm, orb.t_knots, orb.pos[s, d]) for d in range(3)] for s in range(3)])
    n12 = (x[0] - x[1]) / np.linalg.norm(x[0] - x[1])
    perp = np.cross(n12, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp)
    k = np.cos(1.4e-3) * n12 + np.sin(1.4e-3) * perp  # propagation direction; e_r = -k
    lam, beta = float(np.arctan2(-k[1], -k[0])), float(np.arcsin(-k[2]))
    for f in (1e-4, 3e-3):
        src = synth.Source(A=1e-21, f=f, fdot=0.0, phi0=0.3, iota=0.7, psi=0.2, lam=lam, beta=beta)
        mixed(ctx, src, N, 25, orbits["flex"])


def test_tile_beyond_staging_capacity_is_refused(ctx, orbits):
    """A mixed tile whose link span would not fit the shared-memory arrays is a range error."""
    with pytest.raises(lr.LRError) as e:
        lr.Plan(ctx, 25, 4096, DT, orbits["flex"].gpu, t0=T0, precision=lr.MIXED, tile=512)
    assert e.value.status == 2


def test_drawn_sources_per_source_error(ctx, orbits):
    """Sources drawn as in the batched workload (f log-uniform 0.1-10 mHz, isotropic)."""
    worst = 0.0
    for src in synth.draw_sources(12, seed=77, A=1e-22):
        worst = max(worst, mixed(ctx, src, 16384, 25, orbits["flex"]))
    assert worst < RELMX


def test_delay_crossing_a_whole_sample_inside_a_tile(ctx):
    """A link delay that sweeps across dt inside a tile: chained delays change their integer
    sample index mid-tile, which the kernel handles with exact (not expanded) weights."""
    N = 20000
    tk = synth.knot_grid(-2e6, N * DT + 2e6, 1e5)
    pos = synth.static_triangle(tk)
    dl = np.full((6, len(tk)), 2.5e9 / synth.C_LIGHT)
    tc = 0.5 * N * DT
    dl[0] = DT + 0.2 * (tk - tc) / (N * DT)      # L12 crosses one sample at tc
    dl[5] = 0.5 * DT + 0.3 * (tk - tc) / (N * DT)  # L21 crosses half a sample, chains cross integers
    orb = synth.Orbit(tk, pos, dl)
    pr = Pair(ctx, orb)
    src = synth.Source(A=1e-21, f=4e-3, fdot=0.0, phi0=0.1, iota=0.3, psi=0.2, lam=2.0, beta=-0.4)
    mixed(ctx, src, N, 25, pr)
    run_case(ctx, src, N, 25, pr)


def test_batched_mixed_matches_single_calls(ctx, orbits):
    lens = np.array([0, 1, 777, 5000, 12345, 300])
    srcs = synth.draw_sources(len(lens), seed=9, A=1e-22)
    p = 25
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
    o = orbits["flex"]
    for precision, rel in ((lr.MIXED, RELMX), (lr.FP64, 1e-12)):
        plan = lr.Plan(ctx, p, 1, DT, o.gpu, t0=T0, precision=precision)
        xyz = host(plan.response_batched(torch.tensor(h_off, device="cuda:0"), torch.tensor(out_off, device="cuda:0"),
                                         dev(t0h), dev(skyarr), dev(hp), dev(hc)))
        plan.check()
        for s, src in enumerate(srcs):
            N = int(lens[s])
            if N == 0:
                continue
            got = xyz[3 * out_off[s]:3 * out_off[s + 1]].reshape(3, N)
            args = (p, 2, DT, T0, N, o.orc, o.orc, hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]], t0h[s],
                    src.lam, src.beta, src.psi)
            assert_close(got, oracle.response(*args), oracle.response(*args, absval=True), p + 1, rel, f"source {s}")


def test_one_year_mixed_sampled(ctx):
    N, p = synth.ONE_YEAR_SAMPLES, 25
    src = synth.draw_sources(1, seed=1, A=1e-21)[0]
    o = Pair(ctx, synth.orbit_flexing(-3e5, N * DT + 3e5))
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, o.gpu, t0=T0, precision=lr.MIXED)
    got = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
    plan.check()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 1, 2, 255, 256, 257, N // 2, N - 2, N - 1], rng.integers(0, N, 291)]))
    args = (p, 2, DT, T0, N, o.orc, o.orc, hp, hc, t0h, src.lam, src.beta, src.psi, idx)
    assert_close(got[:, idx], oracle.response_at(*args), oracle.response_at(*args, absval=True), p + 1, RELMX)


@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("f", [1e-4, 3e-3])
@pytest.mark.parametrize("kind", ["response", "tdi"])
def test_nested_delays(ctx, orbits, gen, f, kind):
    """Nested chained delays (t_k = t_{k-1} - L(t_{k-1})) against the oracle's nested form."""
    src = synth.Source(A=1e-21, f=f, fdot=1e-17, phi0=0.3, iota=0.7, psi=0.4, lam=1.0, beta=0.3)
    mixed(ctx, src, 30000, 25, orbits["flex"], gen=gen, delay_mode=lr.DELAY_NESTED, kind=kind)


def test_nested_and_summed_differ_as_in_the_oracle(ctx, orbits):
    """At 1 mHz on the flexing orbit the nested and summed responses differ by ~3e-7 relative,
    about 15 times the mixed path's error: each mode must land on its own form."""
    src = synth.Source(A=1e-21, f=1e-3, fdot=1e-17, phi0=0.3, iota=0.7, psi=0.4, lam=1.0, beta=0.3)
    N, p = 30000, 25
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    o = orbits["flex"]
    out = {}
    for dm in (lr.DELAY_SUM, lr.DELAY_NESTED):
        plan = lr.Plan(ctx, p, N, DT, o.gpu, t0=T0, delay_mode=dm, precision=lr.MIXED)
        out[dm] = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
        plan.check()
    args = (p, 2, DT, T0, N, o.orc, o.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
    nested = oracle.response(*args, delay_mode=oracle.DELAY_NESTED)
    summed = oracle.response(*args)
    # each mode lands much closer to its own oracle form than to the other one
    for got, own, other in ((out[lr.DELAY_NESTED], nested, summed), (out[lr.DELAY_SUM], summed, nested)):
        assert np.linalg.norm(got - own) < np.linalg.norm(got - other) / 3
