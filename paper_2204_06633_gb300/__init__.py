"""Python binding of liblisaresp, the GB300-native generic LISA response library
(arXiv:2204.06633: projection of h+, hx onto the six links and TDI X, Y, Z).

This module only marshals arguments: every step of the response runs in the library's CUDA
kernels (``csrc/``), reached through the C ABI declared in ``include/lisaresp.h``.  PyTorch
supplies device memory and streams.  If the compiled library is missing, importing works but
every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblisaresp.so")

FP64, MIXED = 0, 1
DELAY_SUM, DELAY_NESTED = 0, 1
NOT_A_KNOT, NATURAL = 0, 1
LINKS = ("12", "23", "31", "13", "32", "21")

_lib = None


class LRError(RuntimeError):
    def __init__(self, where: str, status: int, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status)} (status {status})"
        super().__init__(msg + (f" {detail}" if detail else ""))


class lr_sky(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("beta", ctypes.c_double), ("psi", ctypes.c_double)]


class lr_gb(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("f0", ctypes.c_double), ("fdot", ctypes.c_double),
                ("fddot", ctypes.c_double), ("phi0", ctypes.c_double), ("iota", ctypes.c_double)]


class lr_time_shard(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("count", ctypes.c_int64), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64)]


class lr_plan_desc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("precision", ctypes.c_int), ("tdi_generation", ctypes.c_int),
                ("delay_mode", ctypes.c_int), ("dt", ctypes.c_double), ("t0", ctypes.c_double),
                ("n", ctypes.c_int64), ("proj_orbit", ctypes.c_void_p), ("tdi_orbit", ctypes.c_void_p),
                ("tile", ctypes.c_int), ("threads", ctypes.c_int)]


_I, _I64, _D, _P = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "lr_strerror": (ctypes.c_char_p, [_I]),
    "lr_version": (_I, []),
    "lr_order_supported": (_I, [_I]),
    "lr_debug_fail_allocations": (_I, [_I]),
    "lr_ctx_create": (_I, [_I, _PP]),
    "lr_ctx_destroy": (_I, [_P]),
    "lr_last_cuda_error": (_I, [_P]),
    "lr_orbit_create": (_I, [_P, _P, _I64, _P, _P, _I, _PP]),
    "lr_orbit_destroy": (_I, [_P]),
    "lr_orbit_delays": (_I, [_P, _P, _I64]),
    "lr_plan_create": (_I, [_P, ctypes.POINTER(lr_plan_desc), _PP]),
    "lr_plan_destroy": (_I, [_P]),
    "lr_required_margin": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "lr_plan_check": (_I, [_P, _P]),
    "lr_project": (_I, [_P, _P, _P, _I64, _D, lr_sky, _P, _P]),
    "lr_tdi": (_I, [_P, _P, _P, _P]),
    "lr_response": (_I, [_P, _P, _P, _I64, _D, lr_sky, _P, _P]),
    "lr_backward": (_I, [_P, _P, _P, _I64, _D, lr_sky, _P, _P, _P, _P, _P]),
    "lr_response_batched": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lr_backward_batched": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lr_response_batched_noalloc": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lr_response_batched_host": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lr_response_batched_graph": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _PP]),
    "lr_graph_launch": (_I, [_P, _P]),
    "lr_graph_destroy": (_I, [_P]),
    "lr_plan_autotune": (_I, [_P, _I64, _I, _P, ctypes.POINTER(_I)]),
    "lr_plan_autotune_batch": (_I, [_P, _I64, _P, _I, _P, ctypes.POINTER(_I)]),
    "lr_choose_order": (_I, [_D, _D, ctypes.POINTER(_I)]),
    "lr_likelihood": (_I, [_P, _P, _P, _I64, _D, lr_sky, _P, _P, _P, _P, _P]),
    "lr_likelihood_batched": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "lr_log_likelihood": (_I, [_P, _P, _P, _I64, _D, lr_sky, _P, _P, _P, _P, _P]),
    "lr_log_likelihood_batched": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "lr_valid_range": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "lr_plan_tile": (_I, [_P, ctypes.POINTER(_I)]),
    "lr_gb_polarisations": (_I, [ctypes.POINTER(lr_gb), _D, _D, _I64, _P, _P, _P]),
    "lr_response_gb": (_I, [_P, lr_gb, lr_sky, _P, _P]),
    "lr_response_gb_batched": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "lr_log_likelihood_gb_batched": (_I, [_P, _I64, _P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "lr_partition_sources": (_I, [_I64, _P, _I, _P, _P]),
    "lr_partition_time": (_I, [_I64, _I64, _I64, _I64, _I, _I, _P]),
    "lr_likelihood_grad": (_I, [_P, _P, _P, _P, _D, _P, _P]),
    "lr_likelihood_grad_batched": (_I, [_P, _I64, _P, _I64, _P, _P, _P, _D, _P, _P]),
}
NOALLOC_MAX_SOURCES = 65536


def library() -> ctypes.CDLL:
    """The loaded liblisaresp (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblisaresp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def strerror(status: int) -> str:
    try:
        return library().lr_strerror(int(status)).decode()
    except Exception:  # library missing while formatting an error
        return "status %d" % status


def _check(where: str, status: int):
    if status != 0:
        raise LRError(where, status)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev64(t: torch.Tensor, name: str, numel: int | None = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def _devi64(t: torch.Tensor, name: str, numel: int) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int64 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def _host(a, dtype, name: str, numel: int | None = None):
    """(pointer, keep-alive object) of a contiguous host array: a CPU torch tensor (pinned or not)
    or anything numpy can view; numpy inputs are converted (copied) only when they must be."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise TypeError(f"{name} must be a host (CPU) array")
        want = torch.float64 if dtype == np.float64 else torch.int64
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous {want} CPU tensor")
        if numel is not None and a.numel() != numel:
            raise ValueError(f"{name} has {a.numel()} elements, expected {numel}")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if numel is not None and arr.size != numel:
        raise ValueError(f"{name} has {arr.size} elements, expected {numel}")
    return arr.ctypes.data, arr


def _gb(gb) -> lr_gb:
    if isinstance(gb, lr_gb):
        return gb
    return lr_gb(*[float(x) for x in gb])


def gb_polarisations(gb, t0: float, dt: float, n: int, device="cuda", stream=None):
    """(h+, hx) of a Galactic binary at t0 + j dt, generated by the library's device generator."""
    hp = torch.empty(int(n), dtype=torch.float64, device=device)
    hc = torch.empty(int(n), dtype=torch.float64, device=device)
    g = _gb(gb)
    _check("lr_gb_polarisations", library().lr_gb_polarisations(ctypes.byref(g), float(t0), float(dt), int(n),
                                                                _dev64(hp, "hp"), _dev64(hc, "hc"),
                                                                _stream_handle(stream)))
    return hp, hc


def _sky(sky) -> lr_sky:
    if isinstance(sky, lr_sky):
        return sky
    lam, beta, psi = sky
    return lr_sky(float(lam), float(beta), float(psi))


class Context:
    def __init__(self, device: int = 0):
        self.device = int(device)
        h = ctypes.c_void_p()
        _check("lr_ctx_create", library().lr_ctx_create(self.device, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lr_ctx_destroy(self._h)
            self._h = None


class Orbit:
    """Spline-interpolated orbit: pos[3][3][n_knots] (m) on uniform knots; delays[6][n_knots] (s)
    or None for the Newtonian light-time solve done by the library."""

    def __init__(self, ctx: Context, t_knots, pos, delays=None, bc: int = NOT_A_KNOT):
        self.ctx = ctx
        self._tk = np.ascontiguousarray(t_knots, dtype=np.float64)
        self._pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(9, -1)
        self._del = None if delays is None else np.ascontiguousarray(delays, dtype=np.float64).reshape(6, -1)
        h = ctypes.c_void_p()
        _check("lr_orbit_create", library().lr_orbit_create(
            ctx.handle, self._tk.ctypes.data, len(self._tk), self._pos.ctypes.data,
            None if self._del is None else self._del.ctypes.data, int(bc), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def delays_at_knots(self):
        out = np.empty((6, len(self._tk)))
        _check("lr_orbit_delays", library().lr_orbit_delays(self._h, out.ctypes.data, len(self._tk)))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lr_orbit_destroy(self._h)
            self._h = None


class Plan:
    """A response configuration: Lagrange degree, precision, TDI generation, delay model,
    output grid (t0 + n*dt, n samples) and the projection / TDI orbits."""

    def __init__(self, ctx: Context, order: int, n: int, dt: float, proj_orbit: Orbit, tdi_orbit: Orbit | None = None,
                 t0: float = 0.0, precision: int = FP64, generation: int = 2, delay_mode: int = DELAY_SUM,
                 tile: int = 0, threads: int = 0):
        self.ctx, self.n, self.order = ctx, int(n), int(order)
        self.proj_orbit = proj_orbit
        self.tdi_orbit = tdi_orbit if tdi_orbit is not None else proj_orbit
        d = lr_plan_desc(int(order), int(precision), int(generation), int(delay_mode), float(dt), float(t0),
                         int(n), proj_orbit.handle.value, self.tdi_orbit.handle.value, int(tile), int(threads))
        self.desc = d
        h = ctypes.c_void_p()
        _check("lr_plan_create", library().lr_plan_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lr_plan_destroy(self._h)
            self._h = None

    def required_margin(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check("lr_required_margin", library().lr_required_margin(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    @property
    def tile(self) -> int:
        """Output samples per CTA tile in use."""
        t = ctypes.c_int()
        _check("lr_plan_tile", library().lr_plan_tile(self._h, ctypes.byref(t)))
        return t.value

    def valid_range(self):
        """(first, last): the outputs whose TDI stencils lie inside [0, n) (inclusive bounds)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check("lr_valid_range", library().lr_valid_range(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def check(self, stream=None):
        """Waits for the stream and raises if a kernel recorded a fault."""
        _check("lr_plan_check", library().lr_plan_check(self._h, _stream_handle(stream)))

    def _out(self, out, shape, like):
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device=like.device)
        return out

    def project(self, hp, hc, t0h, sky, y=None, stream=None):
        y = self._out(y, (6, self.n), hp)
        _check("lr_project", library().lr_project(
            self._h, _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), hp.numel(), float(t0h), _sky(sky),
            _dev64(y, "y", 6 * self.n), _stream_handle(stream)))
        return y

    def tdi(self, y, xyz=None, stream=None):
        xyz = self._out(xyz, (3, self.n), y)
        _check("lr_tdi", library().lr_tdi(self._h, _dev64(y, "y", 6 * self.n), _dev64(xyz, "xyz", 3 * self.n),
                                          _stream_handle(stream)))
        return xyz

    def response(self, hp, hc, t0h, sky, xyz=None, stream=None):
        xyz = self._out(xyz, (3, self.n), hp)
        _check("lr_response", library().lr_response(
            self._h, _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), hp.numel(), float(t0h), _sky(sky),
            _dev64(xyz, "xyz", 3 * self.n), _stream_handle(stream)))
        return xyz

    def response_gb(self, gb, sky, xyz=None, stream=None):
        """Fused response of a Galactic binary generated on the device: gb = (A, f0, fdot, fddot,
        phi0, iota), sky = (lambda, beta, psi); X, Y, Z over the plan's span."""
        xyz = xyz if xyz is not None else torch.empty((3, self.n), dtype=torch.float64, device="cuda")
        _check("lr_response_gb", library().lr_response_gb(self._h, _gb(gb), _sky(sky), _dev64(xyz, "xyz", 3 * self.n),
                                                          _stream_handle(stream)))
        return xyz

    def response_gb_batched(self, out_off, gb, sky, xyz=None, stream=None):
        """out_off int64 CUDA [S+1]; gb float64 CUDA [S][6] (A, f0, fdot, fddot, phi0, iota);
        sky float64 CUDA [S][3]."""
        S = sky.numel() // 3
        total = int(out_off[-1].item()) if xyz is None else xyz.numel() // 3
        xyz = self._out(xyz, (3 * total,), sky)
        _check("lr_response_gb_batched", library().lr_response_gb_batched(
            self._h, S, _devi64(out_off, "out_off", S + 1), _dev64(gb, "gb", 6 * S), _dev64(sky, "sky", 3 * S),
            _dev64(xyz, "xyz"), _stream_handle(stream)))
        return xyz

    def log_likelihood_gb_batched(self, out_off, gb, sky, data, weights=(1.0, 1.0, 1.0), xyz=None, out=None,
                                  stream=None):
        """Per-source <d|h> - <h|h>/2 of generated Galactic binaries, float64 CUDA [S]."""
        S = sky.numel() // 3
        n_total = data.numel() // 3
        out = self._out(out, (S,), sky)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_log_likelihood_gb_batched", library().lr_log_likelihood_gb_batched(
            self._h, S, _devi64(out_off, "out_off", S + 1), _dev64(gb, "gb", 6 * S), _dev64(sky, "sky", 3 * S),
            _dev64(data, "data", 3 * n_total), n_total, ctypes.addressof(w), _dev64(out, "logl", S),
            _dev64(xyz, "xyz", 3 * n_total) if xyz is not None else None, _stream_handle(stream)))
        return out

    def backward(self, hp, hc, t0h, sky, g_xyz, g_hp=None, g_hc=None, g_sky=None, stream=None):
        g_hp = self._out(g_hp, hp.shape, hp)
        g_hc = self._out(g_hc, hc.shape, hc)
        g_sky = self._out(g_sky, (3,), hp)
        _check("lr_backward", library().lr_backward(
            self._h, _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), hp.numel(), float(t0h), _sky(sky),
            _dev64(g_xyz, "g_xyz", 3 * self.n), _dev64(g_hp, "g_hp", hp.numel()), _dev64(g_hc, "g_hc", hp.numel()),
            _dev64(g_sky, "g_sky", 3), _stream_handle(stream)))
        return g_hp, g_hc, g_sky

    def response_batched(self, h_off, out_off, t0h, sky, hp, hc, xyz=None, stream=None):
        """h_off, out_off: int64 CUDA [S+1]; t0h: float64 CUDA [S]; sky: float64 CUDA [S][3]."""
        S = t0h.numel()
        total = int(out_off[-1].item()) if xyz is None else xyz.numel() // 3
        xyz = self._out(xyz, (3 * total,), hp)
        _check("lr_response_batched", library().lr_response_batched(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), _dev64(xyz, "xyz"),
            _stream_handle(stream)))
        return xyz

    def likelihood(self, hp, hc, t0h, sky, data, weights=(1.0, 1.0, 1.0), xyz=None, out=None, stream=None):
        """(<d|h>, <h|h>) as a float64 CUDA tensor [2]: the template's A, E, T against `data`
        (float64 CUDA [3][n] in A, E, T), white noise of variance 1/w_c per channel; the fused
        forward forms them tile by tile.  xyz (optional) also receives X, Y, Z."""
        out = self._out(out, (2,), hp)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_likelihood", library().lr_likelihood(
            self._h, _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), hp.numel(), float(t0h), _sky(sky),
            _dev64(data, "data", 3 * self.n), ctypes.addressof(w), _dev64(out, "dh_hh", 2),
            _dev64(xyz, "xyz", 3 * self.n) if xyz is not None else None, _stream_handle(stream)))
        return out

    def log_likelihood(self, hp, hc, t0h, sky, data, weights=(1.0, 1.0, 1.0), xyz=None, out=None, stream=None):
        """<d|h> - <h|h>/2 as a float64 CUDA tensor [1], formed by the library (see likelihood)."""
        out = self._out(out, (1,), hp)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_log_likelihood", library().lr_log_likelihood(
            self._h, _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), hp.numel(), float(t0h), _sky(sky),
            _dev64(data, "data", 3 * self.n), ctypes.addressof(w), _dev64(out, "logl", 1),
            _dev64(xyz, "xyz", 3 * self.n) if xyz is not None else None, _stream_handle(stream)))
        return out

    def log_likelihood_batched(self, h_off, out_off, t0h, sky, hp, hc, data, weights=(1.0, 1.0, 1.0), xyz=None,
                               out=None, stream=None):
        """Per-source <d|h> - <h|h>/2 as float64 CUDA [S] (arguments as likelihood_batched)."""
        S = t0h.numel()
        if data.numel() % 3:
            raise ValueError("data must hold three channel blocks")
        n_total = data.numel() // 3
        out = self._out(out, (S,), hp)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_log_likelihood_batched", library().lr_log_likelihood_batched(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()),
            _dev64(data, "data", 3 * n_total), n_total, ctypes.addressof(w), _dev64(out, "logl", S),
            _dev64(xyz, "xyz", 3 * n_total) if xyz is not None else None, _stream_handle(stream)))
        return out

    def likelihood_batched(self, h_off, out_off, t0h, sky, hp, hc, data, weights=(1.0, 1.0, 1.0), xyz=None,
                           out=None, stream=None):
        """Per-source (<d|h>, <h|h>) as float64 CUDA [S][2]; data packed like the batched xyz
        (float64 CUDA [3 * sum N_s], source s at 3 out_off[s] as [3][N_s], in A, E, T)."""
        S = t0h.numel()
        if data.numel() % 3:
            raise ValueError("data must hold three channel blocks")
        n_total = data.numel() // 3
        out = self._out(out, (S, 2), hp)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_likelihood_batched", library().lr_likelihood_batched(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()),
            _dev64(data, "data", 3 * n_total), n_total, ctypes.addressof(w), _dev64(out, "dh_hh", 2 * S),
            _dev64(xyz, "xyz", 3 * n_total) if xyz is not None else None, _stream_handle(stream)))
        return out

    def likelihood_grad(self, xyz, data, weights=(1.0, 1.0, 1.0), scale=1.0, g_xyz=None, stream=None):
        """d(<d|h> - <h|h>/2)/d(X, Y, Z) times scale, float64 CUDA [3][n], from the template's X, Y, Z
        and the data in A, E, T (both float64 CUDA [3][n])."""
        g_xyz = self._out(g_xyz, (3, self.n), xyz)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_likelihood_grad", library().lr_likelihood_grad(
            self._h, _dev64(xyz, "xyz", 3 * self.n), _dev64(data, "data", 3 * self.n), ctypes.addressof(w),
            float(scale), _dev64(g_xyz, "g_xyz", 3 * self.n), _stream_handle(stream)))
        return g_xyz

    def likelihood_grad_batched(self, out_off, xyz, data, weights=(1.0, 1.0, 1.0), scale=1.0, g_xyz=None,
                                stream=None):
        """Batched likelihood_grad: xyz, data, g_xyz packed like the batched X, Y, Z."""
        S = out_off.numel() - 1
        if xyz.numel() % 3:
            raise ValueError("xyz must hold three channel blocks")
        g_xyz = self._out(g_xyz, (xyz.numel(),), xyz)
        w = (ctypes.c_double * 3)(*[float(x) for x in weights])
        _check("lr_likelihood_grad_batched", library().lr_likelihood_grad_batched(
            self._h, S, _devi64(out_off, "out_off", S + 1), xyz.numel() // 3, _dev64(xyz, "xyz"),
            _dev64(data, "data", xyz.numel()),
            ctypes.addressof(w), float(scale), _dev64(g_xyz, "g_xyz", xyz.numel()), _stream_handle(stream)))
        return g_xyz

    def response_batched_host(self, h_off, out_off, t0h, sky, hp, hc, xyz=None, stream=None):
        """The batched response on host arrays (numpy or CPU tensors; page-locked tensors let
        the copies overlap the kernels): chunks of sources are copied in, computed and copied
        out concurrently.  Synchronous; returns xyz (host, float64 [3 * out_off[-1]])."""
        S = len(t0h)
        ho, _k1 = _host(h_off, np.int64, "h_off", S + 1)
        oo, _k2 = _host(out_off, np.int64, "out_off", S + 1)
        total = int(out_off[-1])
        if xyz is None:
            xyz = np.empty(3 * total)
        xo, _k3 = _host(xyz, np.float64, "xyz", 3 * total)
        if isinstance(xyz, np.ndarray) and xo != xyz.ctypes.data:
            raise ValueError("xyz must be a contiguous float64 array")
        t0, _k4 = _host(t0h, np.float64, "t0h", S)
        sk, _k5 = _host(sky, np.float64, "sky", 3 * S)
        hpp, _k6 = _host(hp, np.float64, "hp")
        hcp, _k7 = _host(hc, np.float64, "hc", len(hp) if not isinstance(hp, torch.Tensor) else hp.numel())
        _check("lr_response_batched_host", library().lr_response_batched_host(
            self._h, S, ho, oo, t0, sk, hpp, hcp, xo, _stream_handle(stream)))
        return xyz

    def autotune(self, n_samples: int, use_cache: bool = True, stream=None) -> int:
        """Time candidate tile sizes on a synthetic series and keep the fastest; returns it."""
        t = ctypes.c_int(0)
        _check("lr_plan_autotune", library().lr_plan_autotune(self._h, int(n_samples), 1 if use_cache else 0,
                                                              _stream_handle(stream), ctypes.byref(t)))
        self.desc.tile = t.value
        return t.value

    def autotune_batch(self, lengths, use_cache: bool = True, stream=None) -> int:
        """Time candidate tile sizes on a synthetic batch with these source lengths' distribution and
        keep the fastest; returns it."""
        ln = np.ascontiguousarray(lengths, dtype=np.int64)
        t = ctypes.c_int(0)
        _check("lr_plan_autotune_batch", library().lr_plan_autotune_batch(
            self._h, len(ln), ln.ctypes.data, 1 if use_cache else 0, _stream_handle(stream), ctypes.byref(t)))
        self.desc.tile = t.value
        return t.value

    def response_batched_graph(self, h_off, out_off, t0h, sky, hp, hc, xyz):
        """Capture the batched call into a replayable CUDA graph (fixed pointers)."""
        S = t0h.numel()
        h = ctypes.c_void_p()
        _check("lr_response_batched_graph", library().lr_response_batched_graph(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), _dev64(xyz, "xyz"),
            ctypes.byref(h)))
        return Graph(h, keep=(h_off, out_off, t0h, sky, hp, hc, xyz, self))

    def response_batched_noalloc(self, h_off, out_off, t0h, sky, hp, hc, xyz, stream=None):
        """lr_response_batched without any device allocation inside the call (the tile table
        lives in a fixed device array, S <= NOALLOC_MAX_SOURCES); `xyz` must be preallocated.
        Calls that overlap on the GPU share that array and race."""
        S = t0h.numel()
        _check("lr_response_batched_noalloc", library().lr_response_batched_noalloc(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), _dev64(xyz, "xyz"),
            _stream_handle(stream)))
        return xyz

    def backward_batched(self, h_off, out_off, t0h, sky, hp, hc, g_xyz, g_hp=None, g_hc=None, g_sky=None,
                         stream=None):
        S = t0h.numel()
        g_hp = self._out(g_hp, hp.shape, hp)
        g_hc = self._out(g_hc, hc.shape, hc)
        g_sky = self._out(g_sky, (S, 3), hp)
        _check("lr_backward_batched", library().lr_backward_batched(
            self._h, S, _devi64(h_off, "h_off", S + 1), _devi64(out_off, "out_off", S + 1), _dev64(t0h, "t0h", S),
            _dev64(sky, "sky", 3 * S), _dev64(hp, "hp"), _dev64(hc, "hc", hp.numel()), _dev64(g_xyz, "g_xyz"),
            _dev64(g_hp, "g_hp", hp.numel()), _dev64(g_hc, "g_hc", hp.numel()), _dev64(g_sky, "g_sky", 3 * S),
            _stream_handle(stream)))
        return g_hp, g_hc, g_sky


def partition_sources(lengths, ranks: int):
    """(rank_of int32 [S], load int64 [ranks]): the library's length-balanced deal of independent
    sources over ranks (identical on every rank)."""
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    rank_of = np.empty(len(ln), dtype=np.int32)
    load = np.empty(int(ranks), dtype=np.int64)
    _check("lr_partition_sources", library().lr_partition_sources(len(ln), ln.ctypes.data, int(ranks),
                                                                  rank_of.ctypes.data, load.ctypes.data))
    return rank_of, load


def partition_time(n: int, halo_left: int, halo_right: int, align: int, ranks: int, rank: int) -> lr_time_shard:
    """The library's time split of one source's outputs [0, n): rank `rank` owns [first, first + count)
    and computes the span [lo, hi)."""
    out = lr_time_shard()
    _check("lr_partition_time", library().lr_partition_time(int(n), int(halo_left), int(halo_right), int(align),
                                                            int(ranks), int(rank), ctypes.byref(out)))
    return out


def choose_order(f_dt: float, tol: float) -> int:
    """Smallest compiled Lagrange order whose read of a sinusoid at f_dt cycles per sample is within
    tol (see lr_choose_order)."""
    o = ctypes.c_int(0)
    _check("lr_choose_order", library().lr_choose_order(float(f_dt), float(tol), ctypes.byref(o)))
    return o.value


def order_supported(order: int) -> bool:
    return bool(library().lr_order_supported(int(order)))


class Graph:
    """An instantiated CUDA graph of one batched response call."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep  # the captured buffers must outlive the graph

    def launch(self, stream=None):
        _check("lr_graph_launch", library().lr_graph_launch(self._h, _stream_handle(stream)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lr_graph_destroy(self._h)
            self._h = None


class _Response(torch.autograd.Function):
    """X, Y, Z = R(h+, hx; lambda, beta, psi) with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, hp, hc, sky, plan, t0h):
        s = tuple(float(v) for v in sky.detach().cpu().tolist())
        ctx.plan, ctx.t0h, ctx.sky, ctx.sky_device = plan, t0h, s, sky.device
        ctx.save_for_backward(hp, hc)
        return plan.response(hp.contiguous(), hc.contiguous(), t0h, s)

    @staticmethod
    def backward(ctx, g_xyz):
        hp, hc = ctx.saved_tensors
        g_hp, g_hc, g_sky = ctx.plan.backward(hp.contiguous(), hc.contiguous(), ctx.t0h, ctx.sky,
                                              g_xyz.contiguous())
        return g_hp, g_hc, g_sky.to(ctx.sky_device), None, None


def response(plan: Plan, hp, hc, sky, t0h: float):
    """Differentiable fused response: gradients flow to h+, hx and sky = (lambda, beta, psi)
    (a float64 tensor of 3 values)."""
    if not isinstance(sky, torch.Tensor):
        sky = torch.tensor(sky, dtype=torch.float64, device=hp.device)
    return _Response.apply(hp, hc, sky, plan, t0h)


class _LogLikelihood(torch.autograd.Function):
    """<d|h> - <h|h>/2 over A, E, T (the log-likelihood up to -<d|d>/2) with the fused likelihood
    kernel forward and the likelihood gradient + the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, hp, hc, sky, plan, t0h, data, weights):
        s = tuple(float(v) for v in sky.detach().cpu().tolist())
        xyz = torch.empty((3, plan.n), dtype=torch.float64, device=hp.device)
        logl = plan.log_likelihood(hp.contiguous(), hc.contiguous(), t0h, s, data, weights, xyz=xyz)
        ctx.plan, ctx.t0h, ctx.sky, ctx.weights, ctx.sky_device = plan, t0h, s, weights, sky.device
        ctx.save_for_backward(hp, hc, xyz, data)
        return logl[0]

    @staticmethod
    def backward(ctx, g):
        hp, hc, xyz, data = ctx.saved_tensors
        g_xyz = ctx.plan.likelihood_grad(xyz, data, ctx.weights, scale=float(g))
        g_hp, g_hc, g_sky = ctx.plan.backward(hp.contiguous(), hc.contiguous(), ctx.t0h, ctx.sky, g_xyz)
        return g_hp, g_hc, g_sky.to(ctx.sky_device), None, None, None, None


def log_likelihood(plan: Plan, hp, hc, sky, t0h: float, data, weights=(1.0, 1.0, 1.0)):
    """Differentiable <d|h> - <h|h>/2 (A, E, T channels, white noise of variance 1/w_c): gradients
    flow to h+, hx and sky = (lambda, beta, psi); data is float64 CUDA [3][n] in A, E, T."""
    if not isinstance(sky, torch.Tensor):
        sky = torch.tensor(sky, dtype=torch.float64, device=hp.device)
    return _LogLikelihood.apply(hp, hc, sky, plan, t0h, data, tuple(float(x) for x in weights))
