"""Failure detection without a GPU fault: argument and range errors refused on the host,
injected allocation failures reported as LR_ERR_OOM with the library still usable, and a
device-detected fault (inconsistent batch offsets) reported by lr_plan_check."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402

DT = 10.0
INVALID, RANGE, OOM, NONFINITE, UNSUPPORTED, DEVICE = 1, 2, 3, 6, 7, 8


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def orbit(ctx):
    o = synth.orbit_flexing(-2e6, 2e6)
    return lr.Orbit(ctx, o.t_knots, o.pos, None)


def status_of(fn):
    with pytest.raises(lr.LRError) as e:
        fn()
    return e.value.status


def test_plan_arguments_refused_on_host(ctx, orbit):
    assert status_of(lambda: lr.Plan(ctx, 24, 100, DT, orbit)) == UNSUPPORTED          # even order
    assert status_of(lambda: lr.Plan(ctx, 27, 100, DT, orbit)) == UNSUPPORTED          # not compiled
    assert status_of(lambda: lr.Plan(ctx, 25, 0, DT, orbit)) == INVALID
    assert status_of(lambda: lr.Plan(ctx, 25, 100, -1.0, orbit)) == INVALID
    assert status_of(lambda: lr.Plan(ctx, 25, 100, DT, orbit, generation=3)) == INVALID
    assert status_of(lambda: lr.Plan(ctx, 25, 100, DT, orbit, delay_mode=2)) == INVALID


def test_orbit_arguments_refused_on_host(ctx):
    o = synth.orbit_flexing(-2e6, 2e6)
    bad = o.t_knots.copy()
    bad[3] += 10.0
    assert status_of(lambda: lr.Orbit(ctx, bad, o.pos)) == INVALID                      # non-uniform knots
    pos = o.pos.copy()
    pos[0, 0, 2] = np.nan
    assert status_of(lambda: lr.Orbit(ctx, o.t_knots, pos)) == NONFINITE
    assert status_of(lambda: lr.Orbit(ctx, o.t_knots[:3], o.pos[:, :, :3])) == RANGE    # too few knots
    neg = -np.ones((6, len(o.t_knots)))
    assert status_of(lambda: lr.Orbit(ctx, o.t_knots, o.pos, neg)) == RANGE             # negative delays


def test_call_arguments_refused_on_host(ctx, orbit):
    plan = lr.Plan(ctx, 11, 1000, DT, orbit)
    h = torch.zeros(1200, dtype=torch.float64, device="cuda:0")
    assert status_of(lambda: plan.response(h, h, 1e20, (0.1, 0.2, 0.3))) == RANGE       # absurd time offset
    assert status_of(lambda: plan.response(h, h, -100.0, (float("nan"), 0.2, 0.3))) == NONFINITE


def test_injected_allocation_failures(ctx, orbit):
    lib = lr.library()
    o = synth.orbit_flexing(-2e6, 2e6)
    try:
        lib.lr_debug_fail_allocations(0)
        assert status_of(lambda: lr.Orbit(ctx, o.t_knots, o.pos)) == OOM
        assert status_of(lambda: lr.Plan(ctx, 11, 1000, DT, orbit)) == OOM
        lib.lr_debug_fail_allocations(1)   # the plan's error word succeeds, the batch table fails
        plan = lr.Plan(ctx, 11, 1000, DT, orbit)
        z64 = torch.zeros(3, dtype=torch.int64, device="cuda:0")
        zf = torch.zeros(2, dtype=torch.float64, device="cuda:0")
        zs = torch.zeros(6, dtype=torch.float64, device="cuda:0")
        out = torch.zeros(4, dtype=torch.float64, device="cuda:0")
        assert status_of(lambda: plan.response_batched(z64, z64, zf, zs, zf, zf, out)) == OOM
    finally:
        lib.lr_debug_fail_allocations(-1)
    # the library keeps working once allocations succeed again
    src = synth.config1_source()
    t0h, hp, hc = synth.gb_input(src, 0.0, DT, 1000, 11)
    plan = lr.Plan(ctx, 11, 1000, DT, orbit)
    x = plan.response(torch.tensor(hp, device="cuda:0"), torch.tensor(hc, device="cuda:0"), t0h,
                      (src.lam, src.beta, src.psi))
    plan.check()
    assert torch.isfinite(x).all()


def test_device_detected_fault_is_reported(ctx, orbit):
    """Decreasing output offsets: the tile-table kernel records the fault, skips the source,
    and lr_plan_check reports LR_ERR_DEVICE (then clears it)."""
    plan = lr.Plan(ctx, 11, 1, DT, orbit)
    h_off = torch.tensor([0, 500, 1000], dtype=torch.int64, device="cuda:0")
    out_off = torch.tensor([0, 300, 200], dtype=torch.int64, device="cuda:0")
    t0h = torch.full((2,), -400.0, dtype=torch.float64, device="cuda:0")
    sky = torch.tensor([[0.1, 0.2, 0.3], [0.4, 0.5, 0.6]], dtype=torch.float64, device="cuda:0")
    h = torch.ones(1000, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(3 * 300, dtype=torch.float64, device="cuda:0")
    plan.response_batched(h_off, out_off, t0h, sky, h, h, out)
    with pytest.raises(lr.LRError) as e:
        plan.check()
    assert e.value.status == DEVICE
    plan.check()  # cleared


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_nonfinite_strain_and_data_are_reported(ctx, orbit, precision):
    """A NaN in the strain or an infinity in the likelihood data: the kernels record it and
    lr_plan_check reports LR_ERR_NONFINITE (then clears it); finite inputs stay silent."""
    N, p = 5000, 11
    src = synth.draw_sources(1, seed=4, A=1e-21)[0]
    t0h, hp, hc = synth.gb_input(src, 0.0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, orbit, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    sky = (src.lam, src.beta, src.psi)
    plan.response(d(hp), d(hc), t0h, sky)
    plan.check()
    bad = hp.copy()
    bad[N // 2] = np.nan
    plan.response(d(bad), d(hc), t0h, sky)
    assert status_of(plan.check) == NONFINITE
    plan.check()  # cleared
    data = np.zeros((3, N))
    plan.likelihood(d(hp), d(hc), t0h, sky, d(data))
    plan.check()
    data[1, 17] = np.inf
    plan.likelihood(d(hp), d(hc), t0h, sky, d(data))
    assert status_of(plan.check) == NONFINITE
