#!/usr/bin/env python
"""Benchmark of the generic LISA response (projection onto six links + second-generation TDI).

Workload (the batched configuration the headline metric is quoted on): 1024 Galactic binaries
(f log-uniform 0.1-10 mHz, isotropic sky, A = 1e-22, fdot = 1e-17), each with its own length
N_s uniform in [2^16, 2^20] samples at dt = 10 s, flexing Keplerian orbit splined from a 1e5 s
knot grid, Lagrange order 25, one persistent launch per step.  A step = one batched
projection+TDI-2 pass over the whole batch; the metric is link-samples/s = 6 * sum N_s / time.

Output: one JSON line (rank 0).  `value` is device-resident throughput (inputs already in HBM);
`e2e` the same through the C ABI with host buffers (pinned H2D of h+, hx and D2H of X, Y, Z
inside the timed region).  `--impl reference` times the FP64 CPU oracle instead (a bounded
sample of the same workload, on the host's cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "link-samples/s for projection+TDI-2 (batched mixed vs FP64) at stated rel. error"
DT, T0, ORDER, S_SOURCES = 10.0, 0.0, 25, 1024
# algorithmic work per output sample at order p (T = p + 1 taps): tap multiply-adds 60 T
# (9 unique projection reads x 2 polarisations + 42 TDI reads) = 120 T flops, 51 Lagrange
# weight vectors x ~3 T flops, ~500 flops of orbit splines and geometry
FLOPS_PER_SAMPLE = lambda p: 273 * (p + 1) + 500  # noqa: E731
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (nominal; our DFMA probe measured 1.20)
# FP32 ALU peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per output sample of the fused mixed kernel at order 25 and its
# default tile (340), from one ncu capture of a 16-source batch (114.6 MB read + 121.4 MB written
# / 7 115 014 outputs); the launch traffic is this times the launch's outputs.  Valid only for the
# kernel build it was taken on (profiles/k_mixed_fused_batched16_p25.md).
MIXED_P25_DRAM_BYTES_PER_SAMPLE = 235_981_568 / 7_115_014


def workload(rank: int, world: int, n_sources: int):
    """This rank's share of the job's batch: world * n_sources sources (N_s ~ U[2^16, 2^20], seed 3;
    parameters seed 4) dealt over the ranks by the library's length-balanced partition
    (lr_partition_sources), so the work per GPU stays fixed as ranks are added (weak scaling) and
    one rank runs exactly the 1024-source batch."""
    total = world * n_sources
    lens = synth.ragged_lengths(total, seed=3)
    srcs = synth.draw_sources(total, seed=4, A=1e-22, fdot=1e-17)
    if world == 1:
        return lens, srcs
    import paper_2204_06633_gb300 as lr
    rank_of, _ = lr.partition_sources(lens, world)
    sel = np.flatnonzero(rank_of == rank)
    return lens[sel], [srcs[i] for i in sel]


def build_inputs(lens, srcs, p):
    """Packed h+, hx with each source's input margins, CSR offsets, t0_h and sky."""
    m = synth.input_margin_samples(DT, p)
    nh = lens + 2 * m
    h_off = np.concatenate([[0], np.cumsum(nh)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp = np.empty(h_off[-1])
    hc = np.empty(h_off[-1])
    t0h = np.full(len(lens), T0 - m * DT)
    for s, src in enumerate(srcs):
        t = synth.sample_grid(t0h[s], DT, int(nh[s]))
        a, b = synth.gb_polarisations(src, t)
        hp[h_off[s]:h_off[s + 1]] = a
        hc[h_off[s]:h_off[s + 1]] = b
    sky = np.array([[s.lam, s.beta, s.psi] for s in srcs])
    return h_off, out_off, t0h, sky, hp, hc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_scalar(value: float, op: str, device=None) -> float:
    """max or sum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(samples_local: int, ms_local: float, device=None):
    """Whole-job link-samples/s: every rank processes its own batch (weak scaling), so the job
    moved 6 * (sum of all ranks' samples) in the slowest rank's time."""
    total = reduce_scalar(samples_local, "sum", device)
    ms = reduce_scalar(ms_local, "max", device)
    return 6.0 * total / (ms * 1e-3), ms, total


def oracle_rate(lens, srcs, p, orb, budget_s=12.0):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: whole sources of the
    batch, in batch order, until about budget_s of CPU time (the last one truncated)."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    n_try = 20000
    src = srcs[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, n_try, p)
    t = time.perf_counter()
    oracle.response(p, 2, DT, T0, n_try, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    per_sample = (time.perf_counter() - t) / n_try
    left = budget_s / per_sample
    total, elapsed, used = 0, 0.0, 0
    for n_s, src in zip(lens, srcs):
        n = int(min(n_s, left - total))
        if n < 1000:
            break
        t0h, hp, hc = synth.gb_input(src, T0, DT, n, p)
        t = time.perf_counter()
        oracle.response(p, 2, DT, T0, n, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
        elapsed += time.perf_counter() - t
        total += n
        used += 1
    # the same oracle on one thread, on the start of the first source (about 4 s)
    oracle.set_threads(1)
    n1 = int(max(1000, min(int(lens[0]), 4.0 / (per_sample * cores))))
    src = srcs[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, n1, p)
    t = time.perf_counter()
    oracle.response(p, 2, DT, T0, n1, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
    t1 = time.perf_counter() - t
    oracle.set_threads(cores)
    return {"value": 6 * total / elapsed, "unit": "link-samples/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {used} sources of the batch in order ({total} output samples, the last source "
                      f"truncated to fit), {elapsed:.1f} s, FP64 C oracle, OpenMP over samples",
            "single_thread": {"value": 6 * n1 / t1, "unit": "link-samples/s", "cores": 1,
                              "sample": f"the first {n1} outputs of the first source, {t1:.1f} s"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    lens, srcs = workload(0, 1, S_SOURCES)
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * int(lens.max()) + 3e5)
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = oracle_rate(lens, srcs, ORDER, orb, budget_s=max(2.0, 40.0 / (args.warmup + args.steps)))
        if i >= args.warmup:
            times.append(cb["value"])
    v = statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "link-samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched 1024 Galactic binaries, N_s ~ U[2^16, 2^20], dt 10 s, flexing "
                                   "Keplerian orbit, order 25, TDI-2", "sample": cb["sample"]},
            "cpu_baseline": {"value": v, "unit": "link-samples/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "link-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2204_06633_gb300 as lr

    p = args.order
    lens, srcs = workload(rank, ws, args.sources)
    total_samples = int(lens.sum())
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * int(lens.max()) + 3e5)
    h_off, out_off, t0h, sky, hp, hc = build_inputs(lens, srcs, p)

    ctx = lr.Context(local)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    d_hoff = torch.tensor(h_off, device=dev)
    d_ooff = torch.tensor(out_off, device=dev)
    d_t0h = torch.tensor(t0h, device=dev)
    d_sky = torch.tensor(sky, device=dev)
    d_hp = torch.tensor(hp, device=dev)
    d_hc = torch.tensor(hc, device=dev)
    d_xyz = torch.empty(3 * total_samples, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_scalar(v, "max", dev)

    def timed(plan, steps, warmup, sample_clocks=False):
        """W untimed steps, then K steps bracketed by barrier + synchronize; returns
        (ms per step, max over ranks; per-launch ms of this rank; clock summary)."""
        def step():
            plan.response_batched(d_hoff, d_ooff, d_t0h, d_sky, d_hp, d_hc, d_xyz, stream=stream)

        for _ in range(warmup):
            step()
        plan.check(stream)
        barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        barrier()
        plan.check(stream)
        ms = max_over_ranks(t_start.elapsed_time(t_end)) / steps
        return ms, [a.elapsed_time(b) for a, b in ev], (clk.summary() if clk else None), step

    precision = lr.MIXED if args.precision == "mixed" else lr.FP64
    plan = lr.Plan(ctx, p, 1, DT, o, t0=T0, precision=precision, tile=args.tile)
    tile_source = "given"
    if not args.tile:  # the tile the batch autotuner picks for this batch's length mix
        plan.autotune_batch(lens, use_cache=False, stream=stream)
        tile_source = "lr_plan_autotune_batch on this batch"
    ms_step, launch_ms, clocks, step = timed(plan, args.steps, args.warmup, sample_clocks=True)
    value, ms_step, job_samples = job_throughput(total_samples, ms_step, dev)
    link_samples = 6.0 * job_samples

    # accuracy at the stated precision: sampled outputs of a few sources against the oracle
    parity = None
    if rank == 0 and not args.no_check:
        parity = sampled_error(d_xyz, lens, srcs, out_off, orb, p, 1e-6 if precision == lr.MIXED else 1e-12,
                               exact=precision == lr.FP64)

    # end to end through the host-buffer entry point: pinned host arrays in, X, Y, Z back in host
    # memory; the library pipelines chunks of sources (copy-in, kernel, copy-out overlapped).  The
    # call is synchronous, so the region is timed on the host clock.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        hp_pin, hc_pin = pin(hp), pin(hc)
        hoff_pin, ooff_pin, t0h_pin, sky_pin = pin(h_off), pin(out_off), pin(t0h), pin(sky)
        out_pin = torch.empty(3 * total_samples, dtype=torch.float64).pin_memory()

        def e2e_step():
            plan.response_batched_host(hoff_pin, ooff_pin, t0h_pin, sky_pin, hp_pin, hc_pin, xyz=out_pin,
                                       stream=stream)

        e2e_step()  # first call sizes the pipeline's device slots
        torch.cuda.synchronize()
        barrier()
        n_e2e = max(1, min(args.steps, 3))
        t = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        t = max_over_ranks((time.perf_counter() - t) * 1e3 / n_e2e)
        plan.check(stream)
        h2d = sum(int(x.nbytes) for x in (hp, hc, h_off, out_off, t0h, sky))
        e2e = {"value": link_samples / (t * 1e-3), "unit": "link-samples/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(out_pin.numel() * 8), "ms_per_step": t,
               "api": "lr_response_batched_host (host buffers; chunked copy-in, kernel and copy-out overlapped)"}

    # fused likelihood epilogue on the same batch: A, E, T and the inner products per tile, X, Y, Z
    # not written; the data is the batch's own response (values do not change the work)
    like = None
    if not args.no_like:
        data = d_xyz.clone()
        dhh = torch.empty((args.sources, 2), dtype=torch.float64, device=dev)

        def like_step():
            plan.likelihood_batched(d_hoff, d_ooff, d_t0h, d_sky, d_hp, d_hc, data, out=dhh, stream=stream)

        for _ in range(args.warmup):
            like_step()
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            like_step()
        b.record(stream)
        torch.cuda.synchronize()
        plan.check(stream)
        ms_like = max_over_ranks(a.elapsed_time(b) / args.steps)
        like = {"value": link_samples / (ms_like * 1e-3), "unit": "link-samples/s", "ms_per_step": ms_like,
                "steps": args.steps, "warmup": args.warmup, "ms_response_per_step": ms_step,
                "api": "lr_likelihood_batched (per source <d|h>, <h|h> over A, E, T; X, Y, Z not written)"}
        # the same batch with the Galactic-binary strain generated on chip (no strain input):
        # the response, and the sampler's step (parameters in, one log-likelihood per source out)
        gb_h = np.array([[s.A, s.f, s.fdot, s.fddot_value(), s.phi0, s.iota] for s in srcs])
        d_gb = torch.tensor(gb_h, device=dev)
        logl = torch.empty(args.sources, dtype=torch.float64, device=dev)

        def ev_time(f, n):
            for _ in range(args.warmup):
                f()
            torch.cuda.synchronize()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                f()
            b.record(stream)
            torch.cuda.synchronize()
            plan.check(stream)
            return max_over_ranks(a.elapsed_time(b) / n)

        ms_gen = ev_time(lambda: plan.response_gb_batched(d_ooff, d_gb, d_sky, xyz=d_xyz, stream=stream), args.steps)
        ms_genl = ev_time(lambda: plan.log_likelihood_gb_batched(d_ooff, d_gb, d_sky, data, out=logl, stream=stream),
                          args.steps)
        # end to end: pinned host parameters in, the log-likelihoods back in host memory, each step
        gb_pin = torch.from_numpy(np.ascontiguousarray(gb_h)).pin_memory()
        sky_pin = torch.from_numpy(np.ascontiguousarray(sky)).pin_memory()
        logl_pin = torch.empty(args.sources, dtype=torch.float64).pin_memory()

        def gen_e2e_step():
            d_gb.copy_(gb_pin, non_blocking=True)
            d_sky.copy_(sky_pin, non_blocking=True)
            plan.log_likelihood_gb_batched(d_ooff, d_gb, d_sky, data, out=logl, stream=stream)
            logl_pin.copy_(logl, non_blocking=True)
            stream.synchronize()

        gen_e2e_step()
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            gen_e2e_step()
        ms_gen_e2e = max_over_ranks((time.perf_counter() - t) * 1e3 / args.steps)
        plan.check(stream)
        like["generated_strain"] = {
            "response_ms_per_step": ms_gen, "response_value": link_samples / (ms_gen * 1e-3),
            "loglike_ms_per_step": ms_genl, "loglike_value": link_samples / (ms_genl * 1e-3), "unit": "link-samples/s",
            "api": "lr_response_gb_batched / lr_log_likelihood_gb_batched (Galactic binaries generated on chip)",
            "e2e": {"value": link_samples / (ms_gen_e2e * 1e-3), "unit": "link-samples/s", "ms_per_step": ms_gen_e2e,
                    "h2d_bytes_per_step": int(gb_pin.numel() * 8 + sky_pin.numel() * 8),
                    "d2h_bytes_per_step": int(logl_pin.numel() * 8)}}
        del data

    # the same batch in plain FP64 on the same GPU (the comparison the metric names)
    fp64 = None
    if precision == lr.MIXED and not args.no_fp64:
        plan64 = lr.Plan(ctx, p, 1, DT, o, t0=T0, precision=lr.FP64)
        plan64.autotune_batch(lens, use_cache=False, stream=stream)
        ms64, l64, _, _ = timed(plan64, 2, 1)
        fp64 = {"value": link_samples / (ms64 * 1e-3), "unit": "link-samples/s", "ms_per_step": ms64,
                "tile": plan64.tile,
                "steps": 2, "warmup": 1, "mixed_speedup": ms64 / ms_step,
                "roofline": {"bound": "alu", "achieved": FLOPS_PER_SAMPLE(p) * total_samples /
                             (statistics.mean(l64) * 1e-3) / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                             "unit": "TFLOP/s", "frac": FLOPS_PER_SAMPLE(p) * total_samples /
                             (statistics.mean(l64) * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS}}
        if rank == 0 and not args.no_check:
            fp64["parity"] = sampled_error(d_xyz, lens, srcs, out_off, orb, p, 1e-12, exact=True)
            fp64["rel_error_vs_oracle"] = fp64["parity"]["rel_error_vs_oracle"]

    split = None
    if rank == 0 and not args.no_split:
        split = split_times(lr, ctx, p, dev, stream)
    c5 = None
    if rank == 0 and args.config5:
        del d_hp, d_hc, d_xyz
        torch.cuda.empty_cache()
        c5 = config5_times(lr, ctx, dev, stream, args.config5, with_fp64=not args.no_fp64)

    if rank != 0:
        return
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    flops = FLOPS_PER_SAMPLE(p) * total_samples
    if precision == lr.FP64:
        peak_tflops, src_peak = FP64_NOMINAL_TFLOPS, "GB300 FP64 nominal 1.25 TFLOP/s (own DFMA probe: 1.20)"
    else:
        peak_tflops, src_peak = FP32_PEAK_TFLOPS, ("FP32 ALU peak 152 SM x 128 lanes x 2 flop x 2.07 GHz "
                                                   "(own FFMA probe: 74.9 TFLOP/s)")
    traffic = None
    if precision == lr.MIXED and p == 25 and plan.tile == 340:
        traffic = MIXED_P25_DRAM_BYTES_PER_SAMPLE * total_samples
    roof = {"bound": "alu", "achieved": flops / avg_launch_s / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": flops / avg_launch_s / 1e12 / peak_tflops, "traffic": traffic, "peak_source": src_peak,
            "algorithmic_flops_per_sample": FLOPS_PER_SAMPLE(p),
            "kernel": "k_mixed<T,FUSED>" if precision == lr.MIXED else "k_fused64<T>",
            "timing": "CUDA events around each batched call on its stream (tile-table kernel + fused kernel; "
                      "the fused kernel is 99.9 % of it by the ncu launch list)"}
    line = {"metric": METRIC, "value": value, "unit": "link-samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precision == lr.FP64 else "f32 taps + f64 index",
            "data": "synthetic",
            "config": {"workload": "batched 1024 Galactic binaries, N_s ~ U[2^16, 2^20] (sum %d), dt 10 s, "
                                   "flexing Keplerian orbit (1e5 s knots), order %d, TDI-2, fused projection+TDI, "
                                   "one persistent launch per step" % (total_samples, p),
                       "precision": args.precision, "sources_per_gpu": args.sources,
                       "samples_per_gpu": total_samples, "l2": "inputs (%.1f GB) larger than L2" %
                       ((hp.nbytes + hc.nbytes) / 1e9), "tile": plan.tile, "tile_source": tile_source},
            "rel_error_vs_oracle": parity and parity["rel_error_vs_oracle"],
            "error_over_bound": parity and parity["error_over_bound"], "parity": parity, "roofline": roof, "e2e": e2e, "gpu_launches": (3 if precision == lr.MIXED else 2) * args.steps,
            "clocks": clocks, "fp64": fp64, "split": split, "likelihood": like}
    if c5:
        line["differentiation"] = c5
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = oracle_rate(lens, srcs, p, orb)
        if args.oracle_configs:
            line["cpu_baseline"]["configs_in_full"] = oracle_configs(p)
    print(json.dumps(line), flush=True)


def _time_call(f, stream, reps=5):
    """median of `reps` CUDA-event timings of f() on `stream` after 3 warm-up calls (ms)"""
    import torch
    for _ in range(3):
        f()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def split_times(lr, ctx, p, dev, stream, reps=5):
    """The paper's split on its own workload: one one-year source (N = 3,153,600 at dt = 10 s),
    projection alone (h -> six links), TDI-2 alone (links -> X, Y, Z) and the fused call, in each
    precision; the fused call for Lagrange orders 11 / 25 / 41 (the paper's order experiment); and
    the templates: generic (flexing orbit), equal-arm (constant equal arms: the TDI delays are plan
    constants, which the FP64 kernels read with fixed weights), equal-arm with light-time delays
    (the same constellation on the time-dependent-delay path) and hybrid (flexing orbit for the
    projection, constant equal arms for TDI).  CUDA events on the launching stream, median of
    `reps` after 3 warm-up calls."""
    import torch

    N = 3_153_600
    span = (T0 - 3e5, T0 + DT * N + 3e5)
    orb = synth.orbit_flexing(*span)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    src = synth.draw_sources(1, seed=1, A=1e-21, fdot=1e-17)[0]
    sky = (src.lam, src.beta, src.psi)
    y = torch.empty(6 * N, dtype=torch.float64, device=dev)
    xyz = torch.empty(3 * N, dtype=torch.float64, device=dev)
    out = {"workload": "one source, N = 3,153,600 (one year at dt 10 s), flexing orbit, order %d" % p}
    inputs = {}

    def strain(order):
        if order not in inputs:
            t0h, hp, hc = synth.gb_input(src, T0, DT, N, order)
            inputs[order] = (t0h, torch.tensor(hp, device=dev), torch.tensor(hc, device=dev))
        return inputs[order]

    for name, prec in (("mixed", lr.MIXED), ("fp64", lr.FP64)):
        t0h, d_hp, d_hc = strain(p)
        plan = lr.Plan(ctx, p, N, DT, o, t0=T0, precision=prec)
        calls = {"project": lambda: plan.project(d_hp, d_hc, t0h, sky, y, stream=stream),
                 "tdi": lambda: plan.tdi(y, xyz, stream=stream),
                 "fused": lambda: plan.response(d_hp, d_hc, t0h, sky, xyz, stream=stream)}
        out[name] = {k + "_ms": _time_call(f, stream, reps) for k, f in calls.items()}
        plan.check(stream)
    out["orders_fused_ms"] = {}
    for order in (11, 25, 41):
        t0h, d_hp, d_hc = strain(order)
        res = {}
        for name, prec in (("mixed", lr.MIXED), ("fp64", lr.FP64)):
            plan = lr.Plan(ctx, order, N, DT, o, t0=T0, precision=prec)
            res[name] = _time_call(lambda: plan.response(d_hp, d_hc, t0h, sky, xyz, stream=stream), stream, reps)
            plan.check(stream)
        out["orders_fused_ms"][str(order)] = res
    eq = synth.orbit_equal_arm(*span, constant_arms=True)
    eq_o = lr.Orbit(ctx, eq.t_knots, eq.pos, eq.delays)
    eq_lt = lr.Orbit(ctx, eq.t_knots, eq.pos, None)
    templates = {"generic": (o, o), "equal_arm": (eq_o, eq_o), "equal_arm_lighttime": (eq_lt, eq_lt),
                 "hybrid": (o, eq_o)}
    out["templates_fused_ms"] = {}
    t0h, d_hp, d_hc = strain(p)
    for tname, (po, to) in templates.items():
        res = {}
        for name, prec in (("mixed", lr.MIXED), ("fp64", lr.FP64)):
            plan = lr.Plan(ctx, p, N, DT, po, to, t0=T0, precision=prec)
            res[name] = _time_call(lambda: plan.response(d_hp, d_hc, t0h, sky, xyz, stream=stream), stream, reps)
            plan.check(stream)
        out["templates_fused_ms"][tname] = res
    return out


def config5_times(lr, ctx, dev, stream, n_sources=256, with_fp64=True):
    """The differentiation workload: n_sources one-year sources (N = 3,153,600; parameters drawn
    as for the batch, seed 5), flexing orbit, order 41: the batched forward and the batched
    backward (g_h+, g_hx and the sky-angle gradients of white cotangents) per precision, one
    warm-up and one timed call each (CUDA events).  The strain is generated on the device by the
    library's Galactic-binary generator (the same polarisations the arrays would hold)."""
    import torch

    N, p = 3_153_600, 41
    srcs = synth.draw_sources(n_sources, seed=5, A=1e-22, fdot=1e-17)
    m = synth.input_margin_samples(DT, p)
    nh = N + 2 * m
    S = n_sources
    h_off = torch.arange(S + 1, dtype=torch.int64, device=dev) * nh
    out_off = torch.arange(S + 1, dtype=torch.int64, device=dev) * N
    t0h = torch.full((S,), T0 - m * DT, dtype=torch.float64, device=dev)
    sky = torch.tensor([[s.lam, s.beta, s.psi] for s in srcs], dtype=torch.float64, device=dev)
    hp = torch.empty(S * nh, dtype=torch.float64, device=dev)
    hc = torch.empty(S * nh, dtype=torch.float64, device=dev)
    for s, src in enumerate(srcs):
        a, b = lr.gb_polarisations((src.A, src.f, src.fdot, src.fddot_value(), src.phi0, src.iota), T0 - m * DT, DT,
                                   nh, device=dev, stream=stream)
        hp[s * nh:(s + 1) * nh] = a
        hc[s * nh:(s + 1) * nh] = b
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * N + 3e5)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20220413)
    g = torch.randn(3 * S * N, dtype=torch.float64, device=dev, generator=gen)
    out = {"workload": "%d one-year sources (N = 3,153,600), flexing orbit, order 41, white cotangents" % S}
    for name, prec in (("mixed", lr.MIXED), ("fp64", lr.FP64)):
        if prec == lr.FP64 and not with_fp64:
            continue
        plan = lr.Plan(ctx, p, 1, DT, o, t0=T0, precision=prec)
        args = (h_off, out_off, t0h, sky, hp, hc)
        fwd = lambda: plan.response_batched(*args, stream=stream)  # noqa: E731
        bwd = lambda: plan.backward_batched(*args, g, stream=stream)  # noqa: E731
        res = {}
        for k, f in (("forward_s", fwd), ("backward_s", bwd)):
            f()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = f()
            b.record(stream)
            torch.cuda.synchronize()
            res[k] = a.elapsed_time(b) * 1e-3
            del r
        plan.check(stream)
        res["backward_link_samples_per_s"] = 6 * S * N / res["backward_s"]
        out[name] = res
    return out


def oracle_configs(p=25):
    """The FP64 oracle (as it stands, all host cores) on the small configurations in full:
    config 1 (static triangle, N = 65,536, order 25, forward), config 2 (one flexing-orbit one-year
    source, N = 3,153,600, forward) and config 4 (config 1's source at N = 65,536, forward + adjoint
    against white-noise residuals); seconds and link-samples/s."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    out = {"cores": cores}
    src1 = synth.config1_source()
    for name, N, orbf, src in (("config1", 65536, synth.orbit_static, src1),
                               ("config2", 3_153_600, synth.orbit_flexing,
                                synth.draw_sources(1, seed=1, A=1e-21, fdot=1e-17)[0])):
        orb = orbf(T0 - 3e5, T0 + DT * N + 3e5)
        o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        t = time.perf_counter()
        oracle.response(p, 2, DT, T0, N, o, o, hp, hc, t0h, src.lam, src.beta, src.psi)
        s = time.perf_counter() - t
        out[name] = {"seconds": s, "link_samples_per_s": 6 * N / s, "N": N}
    N = 65536
    orb = synth.orbit_static(T0 - 3e5, T0 + DT * N + 3e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    t0h, hp, hc = synth.gb_input(src1, T0, DT, N, p)
    g = synth.white_noise((3, N), 1.0)
    t = time.perf_counter()
    oracle.response(p, 2, DT, T0, N, o, o, hp, hc, t0h, src1.lam, src1.beta, src1.psi)
    oracle.backward(p, 2, DT, T0, N, o, o, hp, hc, t0h, src1.lam, src1.beta, src1.psi, g)
    s = time.perf_counter() - t
    out["config4_65536"] = {"seconds": s, "link_samples_per_s": 6 * N / s, "N": N, "what": "forward + adjoint"}
    return out


def sampled_error(d_xyz, lens, srcs, out_off, orb, p, tol, n_sources=6, n_idx=60, exact=False):
    """Over a few sources of the batch, sampled X, Y, Z against the FP64 oracle: the largest relative
    L2 error, the largest ratio of the error to its bound (the stated tolerance tol, or the
    rounding-error scale K u ||E|| when that is larger: K = 2 (T + 16), u = 2^-53, E the response
    evaluated by the oracle with |weights|, |coefficients| and |inputs|; low-frequency sources are
    ill-conditioned by 1e4-1e7, so two FP64 programs cannot agree to 1e-12 there) and how many
    sources meet tol outright.  exact=True also compares with the exact value of the oracle's
    algorithm (its binary128 build) and reports the FP64 oracle's own error beside it."""
    import oracle
    o = oracle.Orbit(orb.t_knots, orb.pos, None)
    do_exact = exact and oracle.quad_available()
    delays = o.delays_at_knots() if do_exact else None
    rng = np.random.default_rng(7)
    worst, worst_ratio, meets, n = 0.0, 0.0, 0, 0
    worst_exact = worst_oracle_exact = 0.0
    for s in rng.choice(len(lens), n_sources, replace=False):
        N = int(lens[s])
        idx = np.sort(rng.integers(0, N, n_idx))
        src = srcs[s]
        t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
        args = (p, 2, DT, T0, N, o, o, hp, hc, t0h, src.lam, src.beta, src.psi, idx)
        ref = oracle.response_at(*args)
        scale = oracle.response_at(*args, absval=True)
        got = d_xyz[3 * out_off[s]:3 * out_off[s + 1]].view(3, N)[:, idx].cpu().numpy()
        err = float(np.linalg.norm(got - ref))
        nref = float(np.linalg.norm(ref))
        bound = max(tol * nref, 2 * (p + 17) * 2.0 ** -53 * np.linalg.norm(scale))
        worst = max(worst, err / nref)
        worst_ratio = max(worst_ratio, err / bound)
        meets += err <= tol * nref
        n += 1
        if do_exact:
            q = oracle.response_at_quad(p, 2, DT, T0, N, orb.t_knots, orb.pos, delays, hp, hc, t0h, src.lam,
                                        src.beta, src.psi, idx)
            nq = float(np.linalg.norm(q))
            worst_exact = max(worst_exact, float(np.linalg.norm(got - q)) / nq)
            worst_oracle_exact = max(worst_oracle_exact, float(np.linalg.norm(ref - q)) / nq)
    out = {"rel_error_vs_oracle": worst, "error_over_bound": worst_ratio, "tol": tol, "sources_checked": n,
           "sources_within_tol": int(meets), "outputs_per_source": n_idx}
    if do_exact:
        out["rel_error_vs_exact"] = worst_exact
        out["oracle_fp64_rel_error_vs_exact"] = worst_oracle_exact
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--no-like", action="store_true", help="skip the fused likelihood timing")
    ap.add_argument("--no-split", action="store_true",
                    help="skip the projection / TDI / fused split on one one-year source")
    ap.add_argument("--order", type=int, default=ORDER)
    ap.add_argument("--sources", type=int, default=S_SOURCES)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config5", type=int, default=0, metavar="S",
                    help="also time the differentiation workload (S one-year sources, order 41) forward and backward "
                         "in both precisions (S = 256 is the full workload: ~110 GB of device memory)")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="also time the FP64 oracle on configs 1, 2 and 4 in full (about a minute)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
