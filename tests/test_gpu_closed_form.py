"""GPU TDI against the phasor closed form at many frequencies (constant unequal arms, the
frequency-domain cross-check): for sinusoidal link series y_ij = Re(c_ij e^{i w t}) and constant
delays, X1 and X2 are the hand-derived phasor products of Eqs. tdi1/tdi2 (D_ij -> e^{-i w L_ij}).
Both precisions, both generations, 0.1-10 mHz; the bound is the stated tolerance or twice the
oracle's own interpolation error, whichever is larger."""
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
from _helpers import constant_orbit_from, rel_l2  # noqa: E402
from test_oracle_tdi import L_UNEQUAL, phasor_closed_form  # noqa: E402

N = 2048
INTERIOR = slice(60, N - 30)  # away from the zero-extended ends


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def orbits(ctx):
    pos = synth.static_triangle(np.zeros(1))[:, :, 0]
    tk, pp, dl = constant_orbit_from(pos, L_UNEQUAL, -2e6, 2e6)
    return lr.Orbit(ctx, tk, pp, dl), oracle.Orbit(tk, pp, dl)


@pytest.mark.parametrize("precision,tol", [(lr.FP64, 1e-11), (lr.MIXED, 1e-8)])
@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("f", [1e-4, 3e-4, 1e-3, 3e-3, 1e-2])
def test_tdi_matches_phasor_closed_form(ctx, orbits, precision, tol, gen, f):
    p = 25
    og, oo = orbits
    c = np.random.default_rng(3).normal(size=6) + 1j * np.random.default_rng(4).normal(size=6)
    w = 2 * np.pi * f
    t = synth.sample_grid(T0, DT, N)
    y = np.real(c[:, None] * np.exp(1j * w * t)[None, :])
    ref = np.real(phasor_closed_form(c, L_UNEQUAL, w, gen)[:, None] * np.exp(1j * w * t)[None, :])
    plan = lr.Plan(ctx, p, N, DT, og, t0=T0, generation=gen, precision=precision)
    got = host(plan.tdi(dev(y)))
    plan.check()
    err_oracle = rel_l2(oracle.tdi(p, gen, DT, T0, N, oo, y)[:, INTERIOR], ref[:, INTERIOR])
    err = rel_l2(got[:, INTERIOR], ref[:, INTERIOR])
    assert err <= max(tol, 2 * err_oracle), (err, err_oracle)
