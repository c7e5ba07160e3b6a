"""lr_response_batched_noalloc: the batched forward for callers that may not allocate device
memory once their run has started (its tile table lives in a fixed device array inside the
library).  Its X, Y, Z must equal those of lr_response_batched, call after call, although the
shared array keeps the previous call's contents; the calls run with every library allocation
made to fail and leave the device's free memory unchanged; batches beyond the array's capacity
are refused before anything runs.  Kept in a file collected last so that a failure here leaves
every other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402

DT, T0, P = 10.0, 0.0, 25


def batch(lens, seed):
    srcs = synth.draw_sources(len(lens), seed=seed, A=1e-22)
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
    return (d(h_off, torch.int64), d(out_off, torch.int64), d(t0h), d(sky), d(hp), d(hc)), out_off


def per_source_rel(got, ref, out_off):
    worst = 0.0
    for s in range(len(out_off) - 1):
        a, b = got[3 * out_off[s]:3 * out_off[s + 1]], ref[3 * out_off[s]:3 * out_off[s + 1]]
        if b.numel():
            worst = max(worst, float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
    return worst


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_noalloc_matches_batched_on_consecutive_calls(precision, rel):
    ctx = lr.Context(0)
    orb = synth.orbit_flexing(-2e6, 2e5 * DT + 2e6)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=precision)
    # a larger batch first, then a smaller one: the second call runs on top of the table
    # contents the first one left behind
    lib = lr.library()
    for lens, seed in (([777, 5000, 0, 12345, 300, 65536], 31), ([4096, 1, 2000], 32)):
        args, out_off = batch(lens, seed)
        ref = plan.response_batched(*args)
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        # every library allocation fails while this is armed: the call must not need one
        lib.lr_debug_fail_allocations(0)
        try:
            got = plan.response_batched_noalloc(*args, xyz=out)
            torch.cuda.synchronize()
        finally:
            lib.lr_debug_fail_allocations(-1)
        assert torch.cuda.mem_get_info()[0] == free_before  # and no allocation outside the library
        plan.check()
        assert torch.isfinite(got).all()
        assert per_source_rel(got, ref, out_off) <= rel


def test_noalloc_refuses_batches_beyond_its_capacity():
    ctx = lr.Context(0)
    orb = synth.orbit_static(-2e6, 2e6)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0)
    S = lr.NOALLOC_MAX_SOURCES + 1
    z64 = torch.zeros(S + 1, dtype=torch.int64, device="cuda:0")
    zt = torch.zeros(S, dtype=torch.float64, device="cuda:0")
    zs = torch.zeros(3 * S, dtype=torch.float64, device="cuda:0")
    h = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(lr.LRError) as err:
        plan.response_batched_noalloc(z64, z64, zt, zs, h, h, torch.zeros(8, dtype=torch.float64, device="cuda:0"))
    assert err.value.status == 2  # LR_ERR_RANGE
