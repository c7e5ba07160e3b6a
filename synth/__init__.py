"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module only *generates inputs*: source waveforms, spacecraft positions on a
coarse knot grid, source-parameter draws, ragged batch lengths and noise.  It holds
none of the response arithmetic (no projection, no interpolation, no light-time
solve, no TDI): those live independently in the CUDA library and in the CPU oracle.

Conventions
-----------
* SI units: metres, seconds.  c = 299 792 458 m/s, AU = 149 597 870 700 m.
* Spacecraft positions are returned as ``pos[3 spacecraft][3 xyz][n_knots]``.
* Delays, when given as data (the equal-arm constant case), as ``delays[6][n_knots]``
  in the link order 12, 23, 31, 13, 32, 21 (receiver first).
* A "source" is the monochromatic / slowly chirping Galactic binary of the paper's
  Sec. "Template generation": h+ = A (1+cos^2 i) cos(Phi), hx = 2 A cos i sin(Phi),
  Phi = 2 pi (f t + fdot t^2/2 + fddot t^3/6) + phi0, with fddot = 11 fdot^2 / (3 f).
  These are the un-rotated polarisations; the polarisation angle psi is applied by the
  response itself.
"""
from __future__ import annotations

import dataclasses
import numpy as np

C_LIGHT = 299792458.0
AU = 149597870700.0
YEAR = 31557600.0            # Julian year, used as the orbital period
ARM = 2.5e9                  # nominal arm length (m)
ONE_YEAR_SAMPLES = 3153600   # 365 days at dt = 10 s
LINKS = ("12", "23", "31", "13", "32", "21")


# --------------------------------------------------------------------------- sources
@dataclasses.dataclass
class Source:
    A: float
    f: float
    fdot: float
    phi0: float
    iota: float
    psi: float
    lam: float
    beta: float
    fddot: float | None = None

    def fddot_value(self) -> float:
        if self.fddot is not None:
            return self.fddot
        return 11.0 * self.fdot ** 2 / (3.0 * self.f) if self.f > 0 else 0.0


def config1_source() -> Source:
    """The single fixed source of the 'plain method' workload (f = 3 mHz)."""
    return Source(A=1e-22, f=3e-3, fdot=0.0, phi0=0.0, iota=0.5, psi=0.4, lam=1.0, beta=0.3,
                  fddot=0.0)


def draw_sources(n: int, seed: int, A: float = 1e-22, fdot: float = 1e-17,
                 fmin: float = 1e-4, fmax: float = 1e-2) -> list[Source]:
    """Sources with f log-uniform in [fmin, fmax], isotropic sky, uniform cos(iota),
    psi in [0, pi), phi0 in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        f = float(np.exp(rng.uniform(np.log(fmin), np.log(fmax))))
        lam = float(rng.uniform(0.0, 2 * np.pi))
        beta = float(np.arcsin(rng.uniform(-1.0, 1.0)))
        iota = float(np.arccos(rng.uniform(-1.0, 1.0)))
        psi = float(rng.uniform(0.0, np.pi))
        phi0 = float(rng.uniform(0.0, 2 * np.pi))
        out.append(Source(A=A, f=f, fdot=fdot, phi0=phi0, iota=iota, psi=psi, lam=lam, beta=beta))
    return out


def gb_phase(src: Source, t: np.ndarray) -> np.ndarray:
    fdd = src.fddot_value()
    return 2.0 * np.pi * (src.f * t + 0.5 * src.fdot * t * t + fdd * t * t * t / 6.0) + src.phi0


def gb_polarisations(src: Source, t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """h+, hx of the source at times t (un-rotated, no psi)."""
    ph = gb_phase(src, np.asarray(t, dtype=np.float64))
    ci = np.cos(src.iota)
    return src.A * (1.0 + ci * ci) * np.cos(ph), 2.0 * src.A * ci * np.sin(ph)


def sample_grid(t0: float, dt: float, n: int) -> np.ndarray:
    return t0 + dt * np.arange(n, dtype=np.float64)


def input_margin_samples(dt: float, order: int) -> int:
    """A generous number of extra input samples on each side of the output span: the
    largest light-time shift of a heliocentric constellation (|x|/c < 510 s), one arm,
    and the interpolation stencil."""
    return int(np.ceil((510.0 + 10.0) / dt)) + (order + 1) // 2 + 4


def gb_input(src: Source, t0: float, dt: float, n: int, order: int):
    """Polarisations on the input grid covering the output span plus margins.
    Returns (t0_h, hp, hc)."""
    m = input_margin_samples(dt, order)
    t0_h = t0 - m * dt
    t = sample_grid(t0_h, dt, n + 2 * m)
    hp, hc = gb_polarisations(src, t)
    return t0_h, hp, hc


# --------------------------------------------------------------------------- orbits
def _tilted_plane_basis(phase: float = 0.0):
    """Orthonormal in-plane basis of a plane inclined by 60 degrees to the ecliptic,
    whose normal leans toward -x (the Sun for a constellation near (1 AU, 0, 0))."""
    s, c = np.sin(np.pi / 3), np.cos(np.pi / 3)
    a1 = np.array([0.0, 1.0, 0.0])
    a2 = np.array([-c, 0.0, -s])
    return a1, a2


def static_triangle(t_knots: np.ndarray, arm: float = ARM, phase: float = 0.0) -> np.ndarray:
    """Rigid equilateral triangle (side `arm`) centred at (1 AU, 0, 0) in a plane at
    60 degrees to the ecliptic; spacecraft 1, 2, 3 clockwise seen from +z.  Positions do
    not depend on time."""
    a1, a2 = _tilted_plane_basis()
    r = arm / np.sqrt(3.0)
    centre = np.array([AU, 0.0, 0.0])
    pos = np.empty((3, 3, len(t_knots)))
    for i in range(3):
        ph = phase - 2.0 * np.pi * i / 3.0          # decreasing angle: clockwise from +z
        x = centre + r * (np.cos(ph) * a1 + np.sin(ph) * a2)
        pos[i] = x[:, None]
    return pos


def keplerian_equal_arm(t_knots: np.ndarray, arm: float = ARM, kappa: float = 0.0,
                        lambda0: float = 0.0) -> np.ndarray:
    """First-order (in eccentricity) heliocentric Keplerian constellation whose arms stay
    equal to leading order: radius 1 AU, e = arm / (2 sqrt(3) AU) (= 0.00482), plane at
    60 degrees to the ecliptic.  Textbook form (Cornish & Rubbo 2003, Eqs. 56-57);
    spacecraft 1, 2, 3 ordered clockwise seen from +z."""
    t = np.asarray(t_knots, dtype=np.float64)
    e = arm / (2.0 * np.sqrt(3.0) * AU)
    alpha = 2.0 * np.pi * t / YEAR + kappa
    pos = np.empty((3, 3, len(t)))
    for i in range(3):
        b = -2.0 * np.pi * i / 3.0 + lambda0
        pos[i, 0] = AU * np.cos(alpha) + 0.5 * e * AU * (np.cos(2 * alpha - b) - 3 * np.cos(b))
        pos[i, 1] = AU * np.sin(alpha) + 0.5 * e * AU * (np.sin(2 * alpha - b) - 3 * np.sin(b))
        pos[i, 2] = -np.sqrt(3.0) * e * AU * np.cos(alpha - b)
    return pos


# per-spacecraft breathing of the offsets from the guiding centre; the amplitudes are
# scaled so that the arm lengths flex by about +-1 % over a year
_BREATH_AMP = (0.0141, -0.0113, 0.0085)
_BREATH_PHASE = (0.3, 2.1, 4.4)


def keplerian_flexing(t_knots: np.ndarray, arm: float = ARM, amp_scale: float = 1.0) -> np.ndarray:
    """The equal-arm constellation with each spacecraft's offset from the guiding centre
    rescaled by (1 + a_i sin(2 pi t / yr + phi_i)): a smooth annual breathing that flexes
    the arms by about +-1 %."""
    t = np.asarray(t_knots, dtype=np.float64)
    pos = keplerian_equal_arm(t, arm)
    centre = pos.mean(axis=0)
    out = np.empty_like(pos)
    for i in range(3):
        s = 1.0 + amp_scale * _BREATH_AMP[i] * np.sin(2 * np.pi * t / YEAR + _BREATH_PHASE[i])
        out[i] = centre + (pos[i] - centre) * s[None, :]
    return out


def knot_grid(t_start: float, t_end: float, spacing: float = 1e5, pad: int = 2) -> np.ndarray:
    """Uniform knots covering [t_start, t_end] with `pad` extra knots on each side."""
    k0 = int(np.floor(t_start / spacing)) - pad
    k1 = int(np.ceil(t_end / spacing)) + pad
    return spacing * np.arange(k0, k1 + 1, dtype=np.float64)


def constant_delays(n_knots: int, arm: float = ARM) -> np.ndarray:
    """All six delays equal to arm / c at every knot (the equal-arm constant case)."""
    return np.full((6, n_knots), arm / C_LIGHT)


@dataclasses.dataclass
class Orbit:
    t_knots: np.ndarray
    pos: np.ndarray                  # [3][3][nk]
    delays: np.ndarray | None        # [6][nk] or None (light-time solve by the response)


def orbit_static(t_start: float, t_end: float, spacing: float = 1e5) -> Orbit:
    tk = knot_grid(t_start, t_end, spacing)
    return Orbit(tk, static_triangle(tk), constant_delays(len(tk)))


def orbit_equal_arm(t_start: float, t_end: float, spacing: float = 1e5,
                    constant_arms: bool = False) -> Orbit:
    tk = knot_grid(t_start, t_end, spacing)
    return Orbit(tk, keplerian_equal_arm(tk), constant_delays(len(tk)) if constant_arms else None)


def orbit_flexing(t_start: float, t_end: float, spacing: float = 1e5) -> Orbit:
    tk = knot_grid(t_start, t_end, spacing)
    return Orbit(tk, keplerian_flexing(tk), None)


# --------------------------------------------------------------------------- batches
def ragged_lengths(n: int, seed: int, lo: int = 1 << 16, hi: int = 1 << 20) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n, dtype=np.int64)


def white_noise(shape, sigma: float, seed: int = 20220413) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).normal(0.0, sigma, size=shape)


def random_series(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, scale, size=n)
