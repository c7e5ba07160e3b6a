"""lr_response_batched_host: the batched response on host buffers, pipelined in chunks of
sources over three streams, must give exactly the device-resident batched results."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0  # noqa: E402


def batch(S, seed, p):
    lens = synth.ragged_lengths(S, seed=seed, lo=3000, hi=40000)
    srcs = synth.draw_sources(S, seed=seed + 1, A=1e-22, fdot=1e-17)
    m = synth.input_margin_samples(DT, p)
    nh = lens + 2 * m
    h_off = np.concatenate([[0], np.cumsum(nh)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp, hc = np.empty(h_off[-1]), np.empty(h_off[-1])
    t0h = np.full(S, T0 - m * DT)
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, synth.sample_grid(t0h[s], DT, int(nh[s])))
        hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]] = a, b
    sky = np.array([[x.lam, x.beta, x.psi] for x in srcs])
    return h_off, out_off, t0h, sky, hp, hc, int(lens.max())


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.mark.parametrize("precision", [lr.MIXED, lr.FP64])
@pytest.mark.parametrize("chunk", [60000, 1, 10 ** 9])
def test_host_pipeline_matches_device_batch(ctx, monkeypatch, precision, chunk):
    """Chunks of ~60k outputs (many chunks, both slots reused), one source per chunk, one chunk."""
    monkeypatch.setenv("LR_PIPELINE_CHUNK_OUTPUTS", str(chunk))
    p = 25
    h_off, out_off, t0h, sky, hp, hc, nmax = batch(23, 11, p)
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * nmax + 3e5)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    plan = lr.Plan(ctx, p, 1, DT, o, t0=T0, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    ref = plan.response_batched(d(h_off), d(out_off), d(t0h), d(sky), d(hp), d(hc)).cpu().numpy()
    plan.check()
    # page-locked tensors (overlapping copies) and plain numpy arrays (serialised copies)
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    got_pinned = plan.response_batched_host(pin(h_off), pin(out_off), pin(t0h), pin(sky), pin(hp), pin(hc),
                                            xyz=torch.empty(3 * int(out_off[-1]), dtype=torch.float64).pin_memory())
    got_numpy = plan.response_batched_host(h_off, out_off, t0h, sky, hp, hc)
    plan.check()
    assert np.array_equal(got_pinned.numpy(), ref)
    assert np.array_equal(got_numpy, ref)


def test_host_pipeline_refuses_bad_offsets(ctx):
    h_off, out_off, t0h, sky, hp, hc, nmax = batch(4, 3, 25)
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * nmax + 3e5)
    plan = lr.Plan(ctx, 25, 1, DT, lr.Orbit(ctx, orb.t_knots, orb.pos, None), t0=T0, precision=lr.MIXED)
    bad = out_off.copy()
    bad[2], bad[3] = bad[3], bad[2]
    with pytest.raises(lr.LRError) as e:
        plan.response_batched_host(h_off, bad, t0h, sky, hp, hc)
    assert e.value.status == 1
