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
    |coefficients| and |inputs|, K = a bound on the length of the longest accumulation chain)."""
    K = 2 * (T + 16)
    return rel * np.linalg.norm(ref) + K * U64 * np.linalg.norm(scale)


def assert_close(got, ref, scale, T, rel, what=""):
    err = np.linalg.norm(got - ref)
    bound = parity_bound(ref, scale, T, rel)
    relerr = err / np.linalg.norm(ref)
    assert err <= bound, f"{what}: rel L2 {relerr:.3e}, bound {bound / np.linalg.norm(ref):.3e}"
    return relerr
