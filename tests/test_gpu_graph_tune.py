"""CUDA-graph replay of the batched response and the tile autotuner (through the C ABI)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402

DT, T0, P = 10.0, 0.0, 25


def make_batch(lens, seed, scale=1.0):
    srcs = synth.draw_sources(len(lens), seed=seed, A=1e-22 * scale)
    m = synth.input_margin_samples(DT, P)
    lens = np.asarray(lens, dtype=np.int64)
    h_off = np.concatenate([[0], np.cumsum(lens + 2 * m)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp = np.zeros(h_off[-1])
    hc = np.zeros(h_off[-1])
    t0h = np.full(len(lens), T0 - m * DT)
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, synth.sample_grid(t0h[s], DT, int(lens[s] + 2 * m)))
        hp[h_off[s]:h_off[s + 1]] = a
        hc[h_off[s]:h_off[s + 1]] = b
    sky = np.array([[s.lam, s.beta, s.psi] for s in srcs])
    d = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda:0")  # noqa: E731
    return [d(h_off, torch.int64), d(out_off, torch.int64), d(t0h), d(sky), d(hp), d(hc)]


@pytest.fixture(scope="module")
def setup():
    ctx = lr.Context(0)
    orb = synth.orbit_flexing(-2e6, 2e5 * DT + 2e6)
    return ctx, lr.Orbit(ctx, orb.t_knots, orb.pos, None)


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_graph_replay_matches_direct_calls(setup, precision):
    ctx, o = setup
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    lens = [3000, 12000, 777]
    args = make_batch(lens, 41)
    xyz = torch.zeros(3 * sum(lens), dtype=torch.float64, device="cuda:0")
    g = plan.response_batched_graph(*args, xyz)
    for seed, scale in ((41, 1.0), (42, 3.0)):
        new = make_batch(lens, seed, scale)
        args[4].copy_(new[4])          # new strain values, same buffers
        args[5].copy_(new[5])
        args[3].copy_(new[3])          # new sky positions
        g.launch()
        torch.cuda.synchronize()
        ref = plan.response_batched(*args)
        plan.check()
        assert torch.equal(xyz, ref)


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_autotune_picks_a_candidate_and_keeps_results(setup, precision, rel, tmp_path):
    ctx, o = setup
    os.environ["LR_AUTOTUNE_CACHE"] = str(tmp_path / "tune.txt")
    N = 200000
    src = synth.draw_sources(1, seed=5, A=1e-21)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    dhp = torch.tensor(hp, device="cuda:0")
    dhc = torch.tensor(hc, device="cuda:0")
    ref_plan = lr.Plan(ctx, P, N, DT, o, t0=T0, precision=precision)
    ref = ref_plan.response(dhp, dhc, t0h, (src.lam, src.beta, src.psi))
    plan = lr.Plan(ctx, P, N, DT, o, t0=T0, precision=precision)
    tile = plan.autotune(N, use_cache=True)
    assert tile > 0
    got = plan.response(dhp, dhc, t0h, (src.lam, src.beta, src.psi))
    plan.check()
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= rel
    # the choice was cached under this GPU / precision / order / length bucket
    text = open(tmp_path / "tune.txt").read()
    assert f"|o{P}|" in text and f" {tile} " in text
    again = lr.Plan(ctx, P, N, DT, o, t0=T0, precision=precision)
    assert again.autotune(N, use_cache=True) == tile


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_graph_survives_a_larger_batch_on_the_same_plan(setup, precision):
    """A larger batched call on the plan after the capture re-allocates the plan's batch tables;
    the graph keeps its own and still replays its batch."""
    ctx, o = setup
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    lens = [2500, 700]
    args = make_batch(lens, 43)
    xyz = torch.zeros(3 * sum(lens), dtype=torch.float64, device="cuda:0")
    g = plan.response_batched_graph(*args, xyz)
    big = make_batch([300] * 64, 44)
    plan.response_batched(*big)          # grows (re-allocates) the plan's batch tables
    g.launch()
    torch.cuda.synchronize()
    ref = plan.response_batched(*args)
    plan.check()
    assert torch.equal(xyz, ref)


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_batch_autotune_picks_a_candidate_and_keeps_results(setup, precision, rel, tmp_path):
    """The batch tuner times candidate tiles on the ragged batch's length mix; the tuned plan's
    results match the default plan's (bit for bit in FP64, where the tile does not enter the
    arithmetic; within the mixed tolerance otherwise) and the choice is cached."""
    ctx, o = setup
    os.environ["LR_AUTOTUNE_CACHE"] = str(tmp_path / "tune.txt")
    lens = [3000, 12000, 777, 65536, 0, 40000]
    args = make_batch(lens, 45)
    ref_plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    ref = ref_plan.response_batched(*args)
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    tile = plan.autotune_batch(lens, use_cache=True)
    assert tile == plan.tile and tile > 0
    got = plan.response_batched(*args)
    plan.check()
    if precision == lr.FP64:
        assert torch.equal(got, ref)
    else:
        assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= rel
    assert "|batch6_" in open(tmp_path / "tune.txt").read()
    again = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    assert again.autotune_batch(lens, use_cache=True) == tile
