"""FP64 CPU oracle of the generic LISA response (arXiv:2204.06633) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  The CUDA library never does, and the oracle shares
no code with it.  The arithmetic lives in ``lr_oracle.c`` (plain C, FP64, each function
citing the paper's section or equation it follows); this module only compiles it with gcc
and marshals numpy arrays.

Array layouts (all float64, C-contiguous):
  positions  pos[3 spacecraft][3 xyz][n_knots]   (m)
  delays     del[6 links][n_knots]               (s), link order 12, 23, 31, 13, 32, 21
  links      y[6][N]                             on the output grid t0 + n dt
  TDI        xyz[3][N]                           X, Y, Z
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblr_oracle.so")
_SRC_Q = os.path.join(_HERE, "lr_oracle_quad.c")
_LIB_Q = os.path.join(_BUILD, "liblr_oracle_quad.so")
_lock = threading.Lock()
_lib = None
_libq = None

NOT_A_KNOT = 0
NATURAL = 1
DELAY_SUM = 0
DELAY_NESTED = 1


def build(force: bool = False) -> str:
    """Compile lr_oracle.c into oracle/_build/liblr_oracle.so (gcc, OpenMP), and the same source
    widened to binary128 (lr_oracle_quad.c) into liblr_oracle_quad.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    global _quad_error
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_Q))
    if force or not os.path.exists(_LIB_Q) or os.path.getmtime(_LIB_Q) < newest:
        tmp = _LIB_Q + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-fvisibility=hidden", "-o", tmp, _SRC_Q,
               "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB_Q)
            _quad_error = None
        else:  # a toolchain without binary128 libm: only the binary128 checks are unavailable
            _quad_error = r.stderr.strip()[-2000:]
    return _LIB


_quad_error = None


def quad_available() -> bool:
    """True when the binary128 build of the oracle exists on this machine."""
    build()
    return os.path.exists(_LIB_Q) and _quad_error is None


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I64, I, P = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "orc_set_threads": (I, [I]),
            "orc_lagrange_weights": (None, [I, D, dp]),
            "orc_lagrange_dweights": (None, [I, D, dp]),
            "orc_lagrange_read": (D, [dp, I64, I64, D, I]),
            "orc_spline_eval_series": (I, [dp, I64, dp, I, dp, I64, dp]),
            "orc_orbit_new": (P, [dp, I64, dp, dp, I, ctypes.POINTER(ctypes.c_int)]),
            "orc_orbit_free": (None, [P]),
            "orc_orbit_eval": (None, [P, D, dp, dp]),
            "orc_orbit_delays_at_knots": (None, [P, dp]),
            "orc_sky_basis": (None, [D, D, dp, dp, dp]),
            "orc_project": (I, [I, D, D, I64, P, dp, dp, I64, D, D, D, D, dp]),
            "orc_project_abs": (I, [I, D, D, I64, P, dp, dp, I64, D, D, D, D, dp]),
            "orc_project_at": (I, [I, D, D, I64, P, dp, dp, I64, D, D, D, D, lp, I64, dp]),
            "orc_tdi": (I, [I, I, I, D, D, I64, P, dp, dp]),
            "orc_tdi_abs": (I, [I, I, I, D, D, I64, P, dp, dp]),
            "orc_response_at": (I, [I, I, I, D, D, I64, P, P, dp, dp, I64, D, D, D, D, lp, I64, dp, I]),
            "orc_tdi_adjoint": (I, [I, I, I, D, D, I64, P, dp, dp]),
            "orc_project_adjoint": (I, [I, D, D, I64, P, I64, D, D, D, D, dp, dp, dp]),
            "orc_sky_gradient": (I, [I, D, D, I64, P, dp, dp, I64, D, D, D, D, dp, dp]),
            "orc_sky_gradient_abs": (I, [I, D, D, I64, P, dp, dp, I64, D, D, D, D, dp, dp]),
            "orc_aet": (None, [dp, I64, dp]),
            "orc_gb_polarisations": (None, [D, D, D, D, D, D, D, D, I64, dp, dp]),
            "orc_like_inner": (None, [dp, dp, I64, dp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _load_quad():
    global _libq
    with _lock:
        if _libq is not None:
            return _libq
    if not quad_available():
        raise RuntimeError(f"the binary128 oracle could not be built: {_quad_error}")
    with _lock:
        lib = ctypes.CDLL(_LIB_Q)
        D, I64, I, P = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        common = [I, I, I, D, D, I64, P, I64, P, P, I, P, P, I64, D, D, D, D]
        lib.orq_set_threads.restype, lib.orq_set_threads.argtypes = I, [I]
        lib.orq_response.restype, lib.orq_response.argtypes = I, common + [P]
        lib.orq_backward.restype, lib.orq_backward.argtypes = I, common + [P, P, P, P]
        lib.orq_response_at.restype, lib.orq_response_at.argtypes = I, common + [P, I64, P]
        lib.orq_gb_polarisations.restype = None
        lib.orq_gb_polarisations.argtypes = [D, D, D, D, D, D, D, D, I64, P, P]
        _libq = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(status: int, what: str):
    if status != 0:
        raise RuntimeError(f"oracle {what} failed with status {status}")


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle; returns the count in effect."""
    return int(_load().orc_set_threads(int(n)))


# ---------------------------------------------------------------- Lagrange
def lagrange_weights(p: int, eps: float) -> np.ndarray:
    w = np.empty(p + 1)
    _load().orc_lagrange_weights(p, float(eps), _dp(w))
    return w


def lagrange_dweights(p: int, eps: float) -> np.ndarray:
    w = np.empty(p + 1)
    _load().orc_lagrange_dweights(p, float(eps), _dp(w))
    return w


def lagrange_read(s, base: int, u: float, p: int) -> float:
    s = _f64(s)
    return float(_load().orc_lagrange_read(_dp(s), len(s), int(base), float(u), p))


# ---------------------------------------------------------------- splines and orbits
def spline_eval(t_knots, y, t, bc: int = NOT_A_KNOT) -> np.ndarray:
    tk, yy, tt = _f64(t_knots), _f64(y), _f64(np.atleast_1d(t))
    out = np.empty(len(tt))
    _check(_load().orc_spline_eval_series(_dp(tk), len(tk), _dp(yy), bc, _dp(tt), len(tt), _dp(out)), "spline")
    return out


class Orbit:
    """Spline-interpolated spacecraft positions and link delays (delays=None: solve the
    Newtonian light-time equation on the knots)."""

    def __init__(self, t_knots, pos, delays=None, bc: int = NOT_A_KNOT):
        lib = _load()
        self.t_knots = _f64(t_knots)
        self._pos = _f64(pos).reshape(9, -1)
        self._del = None if delays is None else _f64(delays).reshape(6, -1)
        st = ctypes.c_int(0)
        self._h = lib.orc_orbit_new(_dp(self.t_knots), len(self.t_knots), _dp(self._pos),
                                    None if self._del is None else _dp(self._del), bc, ctypes.byref(st))
        if not self._h:
            raise RuntimeError(f"oracle orbit construction failed with status {st.value}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_orbit_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def eval(self, t: float):
        """(positions [3][3], delays [6]) at time t."""
        p9, d6 = np.empty(9), np.empty(6)
        _load().orc_orbit_eval(self._h, float(t), _dp(p9), _dp(d6))
        return p9.reshape(3, 3), d6

    def delays_at_knots(self) -> np.ndarray:
        out = np.empty((6, len(self.t_knots)))
        _load().orc_orbit_delays_at_knots(self._h, _dp(out))
        return out


def sky_basis(lam: float, beta: float):
    k, u, v = np.empty(3), np.empty(3), np.empty(3)
    _load().orc_sky_basis(float(lam), float(beta), _dp(k), _dp(u), _dp(v))
    return k, u, v


# ---------------------------------------------------------------- response
def project(p, dt, t0, n, porb: Orbit, hp, hc, t0h, lam, beta, psi, absval: bool = False) -> np.ndarray:
    hp, hc = _f64(hp), _f64(hc)
    y = np.empty((6, n))
    fn = _load().orc_project_abs if absval else _load().orc_project
    _check(fn(p, dt, t0, n, porb.handle, _dp(hp), _dp(hc), len(hp), t0h, lam, beta, psi, _dp(y)), "project")
    return y


def project_at(p, dt, t0, n, porb: Orbit, hp, hc, t0h, lam, beta, psi, idx) -> np.ndarray:
    hp, hc = _f64(hp), _f64(hc)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    y = np.empty((6, len(idx)))
    _check(_load().orc_project_at(p, dt, t0, n, porb.handle, _dp(hp), _dp(hc), len(hp), t0h, lam, beta, psi,
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx), _dp(y)),
           "project_at")
    return y


def tdi(p, gen, dt, t0, n, torb: Orbit, y, delay_mode: int = DELAY_SUM, absval: bool = False) -> np.ndarray:
    y = _f64(y)
    xyz = np.empty((3, n))
    fn = _load().orc_tdi_abs if absval else _load().orc_tdi
    _check(fn(p, gen, delay_mode, dt, t0, n, torb.handle, _dp(y), _dp(xyz)), "tdi")
    return xyz


def response(p, gen, dt, t0, n, porb, torb, hp, hc, t0h, lam, beta, psi, delay_mode: int = DELAY_SUM,
             absval: bool = False) -> np.ndarray:
    """Projection followed by TDI over the whole output span."""
    y = project(p, dt, t0, n, porb, hp, hc, t0h, lam, beta, psi, absval=absval)
    return tdi(p, gen, dt, t0, n, torb, y, delay_mode, absval=absval)


def response_at(p, gen, dt, t0, n, porb, torb, hp, hc, t0h, lam, beta, psi, idx,
                delay_mode: int = DELAY_SUM, absval: bool = False) -> np.ndarray:
    """X, Y, Z at selected output indices (y computed on demand around each)."""
    hp, hc = _f64(hp), _f64(hc)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    xyz = np.empty((3, len(idx)))
    _check(_load().orc_response_at(p, gen, delay_mode, dt, t0, n, porb.handle, torb.handle, _dp(hp), _dp(hc),
                                   len(hp), t0h, lam, beta, psi,
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx), _dp(xyz),
                                   1 if absval else 0), "response_at")
    return xyz


def _quad_common(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, delay_mode, bc):
    tk, ps = _f64(t_knots), _f64(pos).reshape(9, -1)
    dl = None if delays is None else _f64(delays).reshape(6, -1)
    hp, hc = _f64(hp), _f64(hc)
    keep = (tk, ps, dl, hp, hc)
    args = [int(p), int(gen), int(delay_mode), float(dt), float(t0), int(n), tk.ctypes.data, len(tk), ps.ctypes.data,
            None if dl is None else dl.ctypes.data, int(bc), hp.ctypes.data, hc.ctypes.data, len(hp), float(t0h),
            float(lam), float(beta), float(psi)]
    return args, keep


def response_quad(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi,
                  delay_mode: int = DELAY_SUM, bc: int = NOT_A_KNOT) -> np.ndarray:
    """X, Y, Z of ``response`` (one orbit for projection and TDI, given by its knots) computed by
    the same oracle source in binary128 and rounded once to FP64: the exact result of the
    oracle's algorithm on these FP64 inputs, to ~2^-60 relative of the FP64 oracle's own error."""
    args, keep = _quad_common(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, delay_mode, bc)
    xyz = np.empty((3, n))
    _check(_load_quad().orq_response(*args, xyz.ctypes.data), "response_quad")
    del keep
    return xyz


def response_at_quad(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, idx,
                     delay_mode: int = DELAY_SUM, bc: int = NOT_A_KNOT) -> np.ndarray:
    """``response_at`` in binary128 (rounded once to FP64): sampled exact values of long series."""
    args, keep = _quad_common(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, delay_mode, bc)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    xyz = np.empty((3, len(idx)))
    _check(_load_quad().orq_response_at(*args, idx.ctypes.data, len(idx), xyz.ctypes.data), "response_at_quad")
    del keep
    return xyz


def backward_quad(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, gxyz,
                  delay_mode: int = DELAY_SUM, bc: int = NOT_A_KNOT):
    """(g_h+, g_hx, g_sky) of ``backward`` computed in binary128 and rounded once to FP64."""
    args, keep = _quad_common(p, gen, dt, t0, n, t_knots, pos, delays, hp, hc, t0h, lam, beta, psi, delay_mode, bc)
    g = _f64(gxyz).reshape(3, n)
    ghp, ghc, gs = np.empty(len(keep[3])), np.empty(len(keep[3])), np.empty(3)
    _check(_load_quad().orq_backward(*args, g.ctypes.data, ghp.ctypes.data, ghc.ctypes.data, gs.ctypes.data),
           "backward_quad")
    del keep
    return ghp, ghc, gs


def set_threads_quad(n: int) -> int:
    return int(_load_quad().orq_set_threads(int(n)))


# ---------------------------------------------------------------- adjoints
def tdi_adjoint(p, gen, dt, t0, n, torb: Orbit, gxyz, delay_mode: int = DELAY_SUM) -> np.ndarray:
    g = _f64(gxyz)
    gy = np.empty((6, n))
    _check(_load().orc_tdi_adjoint(p, gen, delay_mode, dt, t0, n, torb.handle, _dp(g), _dp(gy)), "tdi_adjoint")
    return gy


def project_adjoint(p, dt, t0, n, porb: Orbit, nh, t0h, lam, beta, psi, gy):
    gy = _f64(gy)
    ghp, ghc = np.empty(nh), np.empty(nh)
    _check(_load().orc_project_adjoint(p, dt, t0, n, porb.handle, nh, t0h, lam, beta, psi, _dp(gy), _dp(ghp),
                                       _dp(ghc)), "project_adjoint")
    return ghp, ghc


def sky_gradient(p, dt, t0, n, porb: Orbit, hp, hc, t0h, lam, beta, psi, gy, absval: bool = False) -> np.ndarray:
    """dLoss/d(lambda, beta, psi) given g_y; absval=True returns the rounding-error scale of
    that sum (every factor by its absolute value), for sizing tolerances."""
    hp, hc, gy = _f64(hp), _f64(hc), _f64(gy)
    g = np.empty(3)
    fn = _load().orc_sky_gradient_abs if absval else _load().orc_sky_gradient
    _check(fn(p, dt, t0, n, porb.handle, _dp(hp), _dp(hc), len(hp), t0h, lam, beta, psi, _dp(gy), _dp(g)),
           "sky_gradient")
    return g


def backward(p, gen, dt, t0, n, porb, torb, hp, hc, t0h, lam, beta, psi, gxyz, delay_mode: int = DELAY_SUM,
             with_scale: bool = False):
    """Gradient of <gxyz, R(h)> with respect to h+, hx and (lambda, beta, psi); with_scale also
    returns the rounding-error scale of the sky-angle gradient."""
    gy = tdi_adjoint(p, gen, dt, t0, n, torb, gxyz, delay_mode)
    ghp, ghc = project_adjoint(p, dt, t0, n, porb, len(hp), t0h, lam, beta, psi, gy)
    gsky = sky_gradient(p, dt, t0, n, porb, hp, hc, t0h, lam, beta, psi, gy)
    if with_scale:
        return ghp, ghc, gsky, sky_gradient(p, dt, t0, n, porb, hp, hc, t0h, lam, beta, psi, gy, absval=True)
    return ghp, ghc, gsky


# ---------------------------------------------------------------- Galactic binary
def gb_polarisations(A, f0, fdot, fddot, phi0, iota, t0, dt, n, quad: bool = False):
    """(h+, hx) [n] of a Galactic binary at t0 + j dt (Sec. "Template generation"; un-rotated, psi
    applied by the response); quad=True evaluates the same formula in binary128."""
    hp, hc = np.empty(int(n)), np.empty(int(n))
    args = [float(A), float(f0), float(fdot), float(fddot), float(phi0), float(iota), float(t0), float(dt), int(n)]
    if quad:
        _load_quad().orq_gb_polarisations(*args, hp.ctypes.data, hc.ctypes.data)
    else:
        _load().orc_gb_polarisations(*args, _dp(hp), _dp(hc))
    return hp, hc


# ---------------------------------------------------------------- likelihood
def aet(xyz) -> np.ndarray:
    """A, E, T of X, Y, Z ([3][n] -> [3][n]); Sec. "Time-delay interferometry"."""
    x = _f64(xyz).reshape(3, -1)
    out = np.empty_like(x)
    _load().orc_aet(_dp(x), x.shape[1], _dp(out))
    return out


def like_inner(xyz, data_aet, w=(1.0, 1.0, 1.0)):
    """(<d|h>, <h|h>) of the template with X, Y, Z `xyz` against data given in A, E, T, white
    noise of variance 1/w_c per channel (Eq. like, time domain)."""
    x = _f64(xyz).reshape(3, -1)
    d = _f64(data_aet).reshape(3, -1)
    if d.shape != x.shape:
        raise ValueError("data and template lengths differ")
    ww = _f64(w).reshape(3)
    out = np.empty(2)
    _load().orc_like_inner(_dp(x), _dp(d), x.shape[1], _dp(ww), _dp(out))
    return float(out[0]), float(out[1])
