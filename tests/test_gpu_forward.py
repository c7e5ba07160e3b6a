"""GPU parity of the forward response (projection, TDI, fused) against the FP64 oracle.

All calls go through the C ABI (liblisaresp.so via the ctypes binding).  Tolerance: relative
L2 1e-12 for the FP64 build, or the rounding-error scale of the computation when the signal
is strongly cancelled by TDI (see tests/_gpu.py)."""
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

REL64 = 1e-12


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


def test_config1_plain_method_fp64(ctx):
    """f = 3 mHz source, static equal-arm triangle, N = 65536, order 25: links and X, Y, Z."""
    src = synth.config1_source()
    porb = Pair(ctx, synth.orbit_static(-2e6, 65536 * DT + 2e6))
    for kind in ("project", "tdi", "response"):
        e = run_case(ctx, src, 65536, 25, porb, kind=kind)
        assert e < REL64, f"{kind}: {e:.3e}"


@pytest.mark.parametrize("precision,rel", [(lr.FP64, REL64), (lr.MIXED, 1e-6)])
def test_config1_against_stored_fixture(ctx, precision, rel):
    """The plain-method workload at the indices of tests/golden/config1_xyz.txt (oracle values
    written by tests/golden/make_golden.py)."""
    import os
    fx = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "config1_xyz.txt"))
    idx, ref = fx[:, 0].astype(np.int64), fx[:, 1:].T
    src = synth.config1_source()
    N, p = 65536, 25
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    o = synth.orbit_static(-2e5, N * DT + 2e5)
    plan = lr.Plan(ctx, p, N, DT, lr.Orbit(ctx, o.t_knots, o.pos, o.delays), t0=T0, precision=precision)
    got = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))[:, idx]
    plan.check()
    assert np.linalg.norm(got - ref) <= rel * np.linalg.norm(ref)


@pytest.mark.parametrize("p", [1, 3, 5, 11, 25, 41])
def test_orders_static_ragged(ctx, p):
    src = synth.config1_source()
    porb = Pair(ctx, synth.orbit_static(-2e6, 2e6))
    run_case(ctx, src, 5000 + 37, p, porb)


@pytest.fixture(scope="module")
def orbits(ctx):
    span = (-2e6, 6e5 * DT + 2e6)
    return {"flex": Pair(ctx, synth.orbit_flexing(*span)), "eq": Pair(ctx, synth.orbit_equal_arm(*span))}


@pytest.mark.parametrize("p", [11, 25, 41])
@pytest.mark.parametrize("template", ["generic", "equal_arm", "hybrid"])
def test_flexing_templates(ctx, orbits, p, template):
    src = synth.draw_sources(1, seed=1, A=1e-21)[0]
    porb = orbits["eq"] if template == "equal_arm" else orbits["flex"]
    torb = orbits["flex"] if template == "generic" else orbits["eq"]
    run_case(ctx, src, 40000 + 123, p, porb, torb)


@pytest.mark.parametrize("kind", ["project", "tdi"])
def test_unfused_stages_on_flexing_orbit(ctx, orbits, kind):
    src = synth.draw_sources(1, seed=2, A=1e-21)[0]
    run_case(ctx, src, 30011, 25, orbits["flex"], kind=kind)


def test_first_generation_and_nested_delays(ctx, orbits):
    src = synth.draw_sources(1, seed=3, A=1e-21)[0]
    run_case(ctx, src, 20000, 25, orbits["flex"], gen=1)
    run_case(ctx, src, 20000, 25, orbits["flex"], delay_mode=lr.DELAY_NESTED)
    run_case(ctx, src, 20000, 25, orbits["flex"], gen=1, delay_mode=lr.DELAY_NESTED)


@pytest.mark.parametrize("N,tile", [(1, 0), (7, 0), (511, 512), (513, 512), (1000, 128), (4096, 1024)])
def test_small_and_ragged_sizes(ctx, orbits, N, tile):
    src = synth.draw_sources(1, seed=4, A=1e-21)[0]
    run_case(ctx, src, N, 25, orbits["flex"], tile=tile)


def test_strain_shorter_than_needed_is_zero_extended(ctx, orbits):
    src = synth.draw_sources(1, seed=5, A=1e-21)[0]
    N, p = 3000, 11
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    hp, hc = hp[40:2000].copy(), hc[40:2000].copy()
    t0h = t0h + 40 * DT + 3.3   # also a non-integer offset between the two grids
    o = orbits["flex"]
    plan = lr.Plan(ctx, p, N, DT, o.gpu, t0=T0)
    got = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
    args = (p, 2, DT, T0, N, o.orc, o.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
    assert_close(got, oracle.response(*args), oracle.response(*args, absval=True), p + 1, REL64)
    plan.check()


def test_zero_input_gives_zero_output(ctx, orbits):
    N = 2048
    plan = lr.Plan(ctx, 25, N, DT, orbits["flex"].gpu)
    z = torch.zeros(N + 200, dtype=torch.float64, device="cuda:0")
    out = plan.response(z, z, -100 * DT, (0.3, 0.2, 0.1))
    assert not torch.any(out)
    plan.check()


def test_one_year_config2_sampled(ctx):
    """N = 3,153,600 (one year at 10 s), flexing orbit on a 1e5 s knot grid, order 25:
    X, Y, Z at 300 sampled outputs (ends, tile boundaries, random) against the oracle."""
    N, p = synth.ONE_YEAR_SAMPLES, 25
    src = synth.draw_sources(1, seed=1, A=1e-21)[0]
    o = Pair(ctx, synth.orbit_flexing(-3e5, N * DT + 3e5))
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, o.gpu, t0=T0)
    got = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
    plan.check()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 1, 2, 511, 512, 513, N // 2, N - 2, N - 1],
                                    rng.integers(0, N, 291)]))
    args = (p, 2, DT, T0, N, o.orc, o.orc, hp, hc, t0h, src.lam, src.beta, src.psi, idx)
    ref = oracle.response_at(*args)
    scale = oracle.response_at(*args, absval=True)
    assert_close(got[:, idx], ref, scale, p + 1, REL64, "one-year sampled")
    assert np.all(np.isfinite(got))
