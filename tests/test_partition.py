"""Multi-GPU partitioning through the library's host-side logic (lr_partition_sources,
lr_partition_time; no GPU needed), and the split runs it defines, on CPU ranks (gloo, world
size 2) with the oracle computing each rank's share:
  - sources dealt to ranks: the gathered per-source outputs equal the unsplit run's;
  - one long source split in time: each rank computes its span (owned outputs widened by the TDI
    reach) and keeps its owned outputs; their union equals the unsplit run bit for bit, the
    ranks' sky-angle gradients all-reduce (three numbers) to the unsplit gradient within its
    rounding scale, and their strain gradients add up to the unsplit one where windows overlap."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import __graft_entry__  # noqa: F401  (repo root on sys.path)
import oracle
import paper_2204_06633_gb300 as lr
import synth
from paper_2204_06633_gb300 import _build

DT, T0 = 10.0, 0.0


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    oracle.build()


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
def test_source_deal_properties(ranks):
    lens = synth.ragged_lengths(1024, seed=3)
    rank_of, load = lr.partition_sources(lens, ranks)
    assert rank_of.min() >= 0 and rank_of.max() < ranks
    for r in range(ranks):
        assert load[r] == lens[rank_of == r].sum()
    assert load.sum() == lens.sum()
    # greedy longest-first: the spread of the loads is at most the longest source
    assert load.max() - load.min() <= lens.max()
    # deterministic
    again, _ = lr.partition_sources(lens, ranks)
    assert np.array_equal(rank_of, again)


def test_source_deal_small_cases():
    rank_of, load = lr.partition_sources([5, 9, 1, 9, 3, 0, 7], 3)
    # 9(#1)->0, 9(#3)->1, 7(#6)->2, 5(#0)->2, 3(#4)->0, 1(#2)->1, 0(#5)->1
    assert rank_of.tolist() == [2, 0, 1, 1, 0, 1, 2]
    assert load.tolist() == [12, 10, 12]
    rank_of, load = lr.partition_sources([], 4)
    assert len(rank_of) == 0 and load.tolist() == [0, 0, 0, 0]
    with pytest.raises(lr.LRError):
        lr.partition_sources([3, -1], 2)
    with pytest.raises(lr.LRError):
        lr.partition_sources([3], 0)


@pytest.mark.parametrize("n,align,ranks", [(1000, 64, 3), (5, 64, 4), (0, 8, 2), (1, 1, 1), (100000, 340, 8),
                                           (4097, 4, 5)])
def test_time_split_properties(n, align, ranks):
    hl, hr = 70, 13
    shards = [lr.partition_time(n, hl, hr, align, ranks, r) for r in range(ranks)]
    nxt = 0
    for s in shards:
        assert s.first == nxt and s.count >= 0
        nxt = s.first + s.count
        if s.count:
            assert s.first % align == 0
            assert 0 <= s.lo <= s.first and s.first + s.count <= s.hi <= n
            assert s.lo == 0 or (s.lo % align == 0 and s.lo <= s.first - hl)
            assert s.hi == n or (s.hi % align == 0 and s.hi >= s.first + s.count + hr)
    assert nxt == n
    counts = [s.count for s in shards]
    assert max(counts) - min(counts) <= align


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _time_case():
    n, p = 1500, 11
    orb = synth.orbit_flexing(T0 - 3e5, T0 + n * DT + 3e5)
    src = synth.draw_sources(1, seed=17, A=1e-21)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
    g = np.random.default_rng(3).standard_normal((3, n))
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    # the TDI reach: 7 link delays plus the stencil on the left, the stencil on the right (the
    # halos lr_valid_range gives)
    lmax = float(o.delays_at_knots().max())
    hl = int(math.ceil(7 * lmax * 1.001 / DT)) + (p - 1) // 2 + 1
    hr = (p - 1) // 2 + 1
    return n, p, orb, o, src, t0h, hp, hc, g, hl, hr


def _worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    oracle.set_threads(1)
    # ---- time split of one source
    n, p, orb, o, src, t0h, hp, hc, g, hl, hr = _time_case()
    sh = lr.partition_time(n, hl, hr, 64, ws, rank)
    m = sh.hi - sh.lo
    t0s = T0 + sh.lo * DT
    # this rank's strain window: the unsplit input shifted by lo samples (same read offsets), the
    # margins around its span replicated from the neighbours' ranges
    margin = synth.input_margin_samples(DT, p)
    win = slice(sh.lo, sh.hi + 2 * margin)
    args = (p, 2, DT, t0s, m, o, o, hp[win], hc[win], t0h + sh.lo * DT, src.lam, src.beta, src.psi)
    xyz = oracle.response(*args)
    own = slice(sh.first - sh.lo, sh.first - sh.lo + sh.count)
    gather = [None] * ws
    dist.all_gather_object(gather, (sh.first, sh.count, xyz[:, own]))
    # adjoint: g on the owned outputs only
    gs = np.zeros((3, m))
    gs[:, own] = g[:, sh.first:sh.first + sh.count]
    ghp, ghc, gsky = oracle.backward(*args, gs)
    tot = torch.tensor(gsky, dtype=torch.float64)
    dist.all_reduce(tot)
    # strain gradients: each rank's window at its place in the unsplit input, overlaps summed
    full_gh = np.zeros((2, len(hp)))
    full_gh[0, win] = ghp
    full_gh[1, win] = ghc
    gh = torch.tensor(full_gh, dtype=torch.float64)
    dist.all_reduce(gh)
    # ---- sources dealt to ranks
    lens = np.array([700, 0, 1, 1200, 333, 950, 64, 2000], dtype=np.int64)
    srcs = synth.draw_sources(len(lens), seed=23, A=1e-21)
    rank_of, _ = lr.partition_sources(lens, ws)
    mine = {}
    for s in np.flatnonzero(rank_of == rank):
        if lens[s] == 0:
            mine[int(s)] = np.zeros((3, 0))
            continue
        th, a, b = synth.gb_input(srcs[s], T0, DT, int(lens[s]), p)
        mine[int(s)] = oracle.response(p, 2, DT, T0, int(lens[s]), o, o, a, b, th, srcs[s].lam, srcs[s].beta,
                                       srcs[s].psi)
    parts = [None] * ws
    dist.all_gather_object(parts, mine)
    if rank == 0:
        out["time"] = gather
        out["gsky"] = tot.numpy()
        out["gh"] = gh.numpy()
        merged = {}
        for d in parts:
            merged.update(d)
        out["sources"] = merged
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_split_runs_match_the_unsplit_run():
    ws, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    n, p, orb, o, src, t0h, hp, hc, g, hl, hr = _time_case()
    args = (p, 2, DT, T0, n, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    # outputs: the owned ranges tile [0, n) and equal the unsplit run bit for bit
    full = oracle.response(*args)
    got = np.zeros_like(full)
    covered = 0
    for first, count, vals in out["time"]:
        got[:, first:first + count] = vals
        covered += count
    assert covered == n
    np.testing.assert_array_equal(got, full)
    # adjoint partials
    ghp, ghc, gsky, scale = oracle.backward(*args, g, with_scale=True)
    assert np.all(np.abs(out["gsky"] - gsky) <= np.maximum(1e-13 * np.abs(gsky), 4 * (p + 17) * 2.0 ** -53 * scale))
    gh = np.stack([ghp, ghc])
    assert np.linalg.norm(out["gh"] - gh) <= 1e-14 * np.linalg.norm(gh)
    # sources
    lens = np.array([700, 0, 1, 1200, 333, 950, 64, 2000], dtype=np.int64)
    srcs = synth.draw_sources(len(lens), seed=23, A=1e-21)
    assert sorted(out["sources"]) == list(range(len(lens)))
    for s in range(len(lens)):
        if lens[s] == 0:
            continue
        th, a, b = synth.gb_input(srcs[s], T0, DT, int(lens[s]), p)
        ref = oracle.response(p, 2, DT, T0, int(lens[s]), o, o, a, b, th, srcs[s].lam, srcs[s].beta, srcs[s].psi)
        np.testing.assert_array_equal(out["sources"][s], ref)
