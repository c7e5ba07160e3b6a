"""Constant TDI delays (the equal-arm template with constant arms, the static triangle): the FP64
kernels read every delayed term with plan-constant weights.  Parity against the oracle for the
fused call and the TDI-only call, TDI generations 1 and 2, summed and nested delays (identical for
constant delays), equal and unequal arms, and the hybrid template (flexing projection orbit)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, Pair, run_case  # noqa: E402

N = 20000


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def eq(ctx):
    return Pair(ctx, synth.orbit_equal_arm(T0 - 3e5, T0 + N * DT + 3e5, constant_arms=True))


@pytest.fixture(scope="module")
def unequal(ctx):
    orb = synth.orbit_equal_arm(T0 - 3e5, T0 + N * DT + 3e5, constant_arms=True)
    orb.delays = orb.delays * np.array([1.0, 1.013, 0.991, 1.0, 0.991, 1.013])[:, None]
    return Pair(ctx, orb)


@pytest.mark.parametrize("p", [11, 25])
@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("dm", [lr.DELAY_SUM, lr.DELAY_NESTED])
def test_constant_delays_fused(ctx, eq, p, gen, dm):
    src = synth.draw_sources(1, seed=60 + p + gen, A=1e-21)[0]
    run_case(ctx, src, N, p, eq, gen=gen, delay_mode=dm)


@pytest.mark.parametrize("kind", ["response", "tdi"])
def test_constant_unequal_arms(ctx, unequal, kind):
    src = synth.draw_sources(1, seed=71, A=1e-21)[0]
    run_case(ctx, src, N, 25, unequal, kind=kind)


def test_hybrid_template(ctx, eq):
    flex = Pair(ctx, synth.orbit_flexing(T0 - 3e5, T0 + N * DT + 3e5))
    src = synth.draw_sources(1, seed=72, A=1e-21)[0]
    run_case(ctx, src, N, 25, flex, torb=eq)
