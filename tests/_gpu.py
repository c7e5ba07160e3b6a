"""GPU-test helpers: build matching library / oracle orbits and compare with the oracle."""
import numpy as np
import torch

import oracle
import paper_2204_06633_gb300 as lr
import synth

U64 = 2.0 ** -53


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def host(t):
    return t.detach().cpu().numpy()


class Pair:
    """The same synthetic orbit in the library and in the oracle."""

    def __init__(self, ctx, orb: synth.Orbit):
        self.orb = orb
        self.gpu = lr.Orbit(ctx, orb.t_knots, orb.pos, orb.delays)
        self.orc = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)


def parity_bound(ref, scale, T, rel):
    """Allowed L2 error: the stated relative tolerance, or the rounding-error scale of the
    computation when that is larger (K * u * ||E||, E = the response evaluated with |weights|,
    |coefficients| and |inputs|, K = a bound on the length of the longest accumulation chain).
    The scale bounds the FP64 oracle's own error against the exact result of its algorithm
    (tests/test_oracle_precision.py), which exceeds 1e-12 at low frequency."""
    K = 2 * (T + 16)
    return max(rel * np.linalg.norm(ref), K * U64 * np.linalg.norm(scale))


def assert_close(got, ref, scale, T, rel, what=""):
    err = np.linalg.norm(got - ref)
    bound = parity_bound(ref, scale, T, rel)
    relerr = err / np.linalg.norm(ref)
    assert err <= bound, f"{what}: rel L2 {relerr:.3e}, bound {bound / np.linalg.norm(ref):.3e}"
    return relerr


DT, T0 = 10.0, 0.0


def sky(src):
    return (src.lam, src.beta, src.psi)


def run_case(ctx, src, N, p, porb, torb=None, gen=2, delay_mode=0, kind="response", tile=0,
             precision=lr.FP64, rel=1e-12):
    """One single-source call through the C ABI against the oracle; returns the relative L2."""
    torb = torb or porb
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, porb.gpu, torb.gpu, t0=T0, generation=gen, delay_mode=delay_mode, tile=tile,
                   precision=precision)
    args = (p, gen, DT, T0, N, porb.orc, torb.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
    if kind == "response":
        got = host(plan.response(dev(hp), dev(hc), t0h, sky(src)))
        ref = oracle.response(*args, delay_mode=delay_mode)
        scale = oracle.response(*args, delay_mode=delay_mode, absval=True)
    elif kind == "project":
        got = host(plan.project(dev(hp), dev(hc), t0h, sky(src)))
        pargs = (p, DT, T0, N, porb.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
        ref = oracle.project(*pargs)
        scale = oracle.project(*pargs, absval=True)
    else:  # tdi on the oracle's link series
        y = oracle.project(p, DT, T0, N, porb.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
        got = host(plan.tdi(dev(y)))
        ref = oracle.tdi(p, gen, DT, T0, N, torb.orc, y, delay_mode)
        scale = oracle.tdi(p, gen, DT, T0, N, torb.orc, np.abs(y), delay_mode, absval=True)
    plan.check()
    return assert_close(got, ref, scale, p + 1, rel, f"{kind} p={p} N={N}")
