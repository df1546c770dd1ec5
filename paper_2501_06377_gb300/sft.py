"""Thin ctypes binding of libsft (include/sft.h).

Argument marshalling only: every step of the SFT path runs in the CUDA
kernels of libsft.so.  Loading fails loudly when the library is missing;
there is no CPU fallback.

Maps may be numpy arrays (host) or torch tensors (host or CUDA), row-major
[ntheta][nphi] in the grid's precision.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re
from dataclasses import dataclass, fields

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsft.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sft.h")

SFT_OK, SFT_ERR_ARG, SFT_ERR_OOM, SFT_ERR_CUDA, SFT_ERR_UNSTABLE, SFT_ERR_TIMEOUT, SFT_ERR_STATE = range(7)
STATUS_NAMES = {0: "SFT_OK", 1: "SFT_ERR_ARG", 2: "SFT_ERR_OOM", 3: "SFT_ERR_CUDA",
                4: "SFT_ERR_UNSTABLE", 5: "SFT_ERR_TIMEOUT", 6: "SFT_ERR_STATE"}
SFT_FP32, SFT_FP64 = 0, 1
ADV_SPACE = {"weno3": 0, "upwind": 1}
ADV_TIME = {"ssprk43": 0, "ssprk33": 1, "fe": 2}
DIFFUSION = {"rkl2": 0, "off": 1, "rkg2": 2}
SPLITTING = {"lie": 0, "strang": 1}


class SFTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class sft_shape(C.Structure):
    _fields_ = [("ntheta", C.c_int32), ("nphi", C.c_int32)]


class sft_flow_params(C.Structure):
    _fields_ = [("d0", C.c_double), ("d2", C.c_double), ("d4", C.c_double),
                ("m1", C.c_double), ("m3", C.c_double), ("m5", C.c_double),
                ("nu", C.c_double), ("alpha_uw", C.c_double), ("cfl_safety", C.c_double),
                ("eps_w", C.c_double), ("adv_space", C.c_int32), ("adv_time", C.c_int32),
                ("diffusion", C.c_int32), ("advection", C.c_int32), ("atten_b0", C.c_double),
                ("splitting", C.c_int32), ("reserved", C.c_int32), ("nu_grid_alpha", C.c_double)]


class sft_rfe_params(C.Structure):
    _fields_ = [("method", C.c_int32), ("origin_given", C.c_int32), ("rate_mx_per_hour", C.c_double),
                ("lifetime_hours", C.c_double), ("seed", C.c_uint64), ("origin_hours", C.c_double)]


class sft_assim_params(C.Structure):
    _fields_ = [("alpha_mu", C.c_double), ("mu_lim", C.c_double), ("lat_lim_deg", C.c_double),
                ("flux_balance", C.c_int32), ("reserved", C.c_int32)]


class sft_diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "flux_signed", "flux_pos", "flux_neg", "flux_pole_n", "flux_pole_s", "area_pole_n",
        "area_pole_s", "brmin", "brmax", "absmin", "dipole_axial", "h1", "h2", "t_hours")] + [
        ("steps", C.c_int64), ("nonfinite", C.c_int64)]


class sft_stats(C.Structure):
    _fields_ = [("global_steps", C.c_int64), ("realization_steps", C.c_int64),
                ("cell_updates", C.c_double), ("adv_cell_stages", C.c_double),
                ("diff_cell_stages", C.c_double), ("kernel_launches", C.c_int64),
                ("graph_launches", C.c_int64), ("diff_ms", C.c_double), ("adv_ms", C.c_double),
                ("diff_launches", C.c_int64), ("adv_launches", C.c_int64),
                ("diff_bytes", C.c_double), ("adv_bytes", C.c_double)]


_lib = None

_SIGS = {
    "sft_create_grid": (C.c_int, [C.POINTER(sft_shape), C.c_int32, C.c_int, C.c_size_t, C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    "sft_destroy": (C.c_int, [C.c_void_p]),
    "sft_set_state": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "sft_get_state": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "sft_set_time": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    "sft_get_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "sft_set_flows": (C.c_int, [C.c_void_p, C.POINTER(sft_flow_params)]),
    "sft_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.POINTER(C.c_int32)]),
    "sft_assimilate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                 C.POINTER(sft_assim_params)]),
    "sft_balance_flux": (C.c_int, [C.c_void_p]),
    "sft_set_rfe": (C.c_int, [C.c_void_p, C.POINTER(sft_rfe_params)]),
    "sft_flux_diagnostics": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(sft_diag)]),
    "sft_get_stats": (C.c_int, [C.c_void_p, C.POINTER(sft_stats)]),
    "sft_reset_stats": (C.c_int, [C.c_void_p]),
    "sft_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "sft_set_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "sft_set_fusion": (C.c_int, [C.c_void_p, C.c_int32]),
    "sft_get_fusion": (C.c_int32, [C.c_void_p]),
    "sft_set_tile_rows": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "sft_get_tile_rows": (C.c_int32, [C.c_void_p, C.c_int32]),
    "sft_set_band_rows": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "sft_get_band_rows": (C.c_int32, [C.c_void_p, C.c_int32]),
    "sft_wave_size": (C.c_int32, [C.c_void_p]),
    "sft_step_plan": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "sft_set_states": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_int32]),
    "sft_get_states": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_int32]),
    "sft_set_times": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "sft_flux_diagnostics_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int,
                                               C.c_double, C.c_void_p, C.POINTER(sft_diag)]),
    "sft_debug_checks": (C.c_int, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint32), C.c_int32]),
    "sft_debug_probe": (C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64]),
    "sft_debug_fail_alloc": (C.c_int, [C.c_int32]),
    "sft_last_error": (C.c_char_p, [C.c_void_p]),
    "sft_abi_version": (C.c_int32, []),
}


def header_functions(path=HEADER, prefix="sft_"):
    """Names of the functions a header (include/sft.h by default) declares."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z0-9_]+)\s*\(", text)))


def load(path=LIB_PATH):
    """Load libsft.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsft.so not built (%s); run paper_2501_06377_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0, a
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(a))


@dataclass
class FlowParams:
    """Python view of sft_flow_params (Eq. dr, Eq. mf; nu in km^2/s)."""
    d0: float = 46.0
    d2: float = -262.0
    d4: float = -379.0
    m1: float = 22.0
    m3: float = 11.0
    m5: float = -28.0
    nu: float = 500.0
    alpha_uw: float = 1.0
    cfl_safety: float = 0.9
    eps_w: float = 0.0
    adv_space: str = "weno3"
    adv_time: str = "ssprk43"
    diffusion: str = "rkl2"
    advection: bool = True
    atten_b0: float = 0.0   # Eq. (flow_attenuation) saturation field in G; 0 = off
    splitting: str = "lie"  # "lie" | "strang" (Sec. 3.5), the same for all realizations
    nu_grid_alpha: float = 0.0  # > 0: grid-based nu of Eq. (diffgrid) (1/hour) instead of nu

    def to_c(self):
        return sft_flow_params(self.d0, self.d2, self.d4, self.m1, self.m3, self.m5, self.nu,
                               self.alpha_uw, self.cfl_safety, self.eps_w,
                               ADV_SPACE[self.adv_space], ADV_TIME[self.adv_time],
                               DIFFUSION[self.diffusion], 1 if self.advection else 0, self.atten_b0,
                               SPLITTING[self.splitting], 0, self.nu_grid_alpha)


@dataclass
class RfeParams:
    """Python view of sft_rfe_params (Sec. 2.4 random flux emergence)."""
    method: int = 2                 # 1: Eq. (rfe_m1), 2: Eq. (rfe_m2)
    rate_mx_per_hour: float = 1e23  # total unsigned flux per hour
    lifetime_hours: float = math.inf
    seed: int = 0
    origin_hours: float = None      # None: the realization's time at set_rfe

    def to_c(self):
        given = self.origin_hours is not None
        return sft_rfe_params(self.method, 1 if given else 0, self.rate_mx_per_hour, self.lifetime_hours,
                              self.seed, float(self.origin_hours) if given else 0.0)


@dataclass
class AssimParams:
    alpha_mu: float = 4.0
    mu_lim: float = 0.1
    lat_lim_deg: float = 90.0
    flux_balance: bool = True

    def to_c(self):
        return sft_assim_params(self.alpha_mu, self.mu_lim, self.lat_lim_deg,
                                1 if self.flux_balance else 0, 0)


class Grid:
    """A batch of realizations (sft_create_grid ... sft_destroy)."""

    def __init__(self, shapes, prec="fp32", hbm_budget=0, stream=None):
        lib = load()
        self.lib = lib
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        self.n_real = len(self.shapes)
        self.prec = prec
        self.dtype = np.float32 if prec == "fp32" else np.float64
        arr = (sft_shape * self.n_real)(*[sft_shape(a, b) for a, b in self.shapes])
        h = C.c_void_p()
        if stream is None:
            s = None
        elif isinstance(stream, int):
            s = stream
        else:
            s = stream.cuda_stream
        st = lib.sft_create_grid(arr, self.n_real, SFT_FP32 if prec == "fp32" else SFT_FP64,
                                 int(hbm_budget), s, C.byref(h))
        if st != SFT_OK:
            raise SFTError(st, lib.sft_last_error(None).decode())
        self.h = h

    # -- helpers ---------------------------------------------------------
    def _check(self, st):
        if st != SFT_OK:
            raise SFTError(st, self.lib.sft_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C-ABI mirrors -----------------------------------------------------
    def sft_set_state(self, r, br):
        p, dev, keep = _ptr(br)
        self._check(self.lib.sft_set_state(self.h, r, C.c_void_p(p), dev))
        del keep

    def set_state(self, r, br):
        if isinstance(br, np.ndarray):
            br = np.ascontiguousarray(br, dtype=self.dtype)
        self.sft_set_state(r, br)

    def get_state(self, r, out=None):
        if not 0 <= r < self.n_real:   # let the library report the bad index
            self._check(self.lib.sft_get_state(self.h, r, None, 0))
        nt, np_ = self.shapes[r]
        if out is None:
            out = np.empty((nt, np_), dtype=self.dtype)
        p, dev, _ = _ptr(out)
        self._check(self.lib.sft_get_state(self.h, r, C.c_void_p(p), dev))
        return out

    def set_time(self, t, r=-1):
        """Set realization r's time (all when r = -1); t may be a sequence of
        per-realization times."""
        if np.ndim(t) == 0:
            self._check(self.lib.sft_set_time(self.h, int(r), float(t)))
        else:
            for i, ti in enumerate(t):
                self._check(self.lib.sft_set_time(self.h, i, float(ti)))

    def _subset(self, idx):
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).ravel())
        return idx, idx.ctypes.data_as(C.POINTER(C.c_int32))

    def set_states(self, idx, maps):
        """sft_set_states: maps[q] (a packed [n, ntheta, nphi] array or tensor)
        into realizations idx[q]."""
        idx, pi = self._subset(idx)
        if isinstance(maps, np.ndarray):
            maps = np.ascontiguousarray(maps, dtype=self.dtype)
        p, dev, keep = _ptr(maps)
        self._check(self.lib.sft_set_states(self.h, len(idx), pi, C.c_void_p(p), dev))
        del keep

    def get_states(self, idx, out):
        """sft_get_states: realizations idx[q] into out[q] (packed, contiguous)."""
        idx, pi = self._subset(idx)
        p, dev, keep = _ptr(out)
        self._check(self.lib.sft_get_states(self.h, len(idx), pi, C.c_void_p(p), dev))
        del keep
        return out

    def set_times(self, idx, t):
        """sft_set_times: realization idx[q] to time t[q] (or all to scalar t)."""
        idx, pi = self._subset(idx)
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), idx.shape))
        self._check(self.lib.sft_set_times(self.h, len(idx), pi, t.ctypes.data_as(C.POINTER(C.c_double))))

    def get_time(self):
        out = (C.c_double * self.n_real)()
        self._check(self.lib.sft_get_time(self.h, out))
        return np.array(out[:])

    def set_flows(self, params):
        if isinstance(params, FlowParams):
            params = [params] * self.n_real
        arr = (sft_flow_params * self.n_real)(*[p.to_c() for p in params])
        self._check(self.lib.sft_set_flows(self.h, arr))

    def set_rfe(self, params):
        """Random flux emergence per realization (a RfeParams, a list of
        them with None for off, or None for off everywhere)."""
        if params is None:
            self._check(self.lib.sft_set_rfe(self.h, None))
            return
        if isinstance(params, RfeParams):
            params = [params] * self.n_real
        arr = (sft_rfe_params * self.n_real)(*[(p or RfeParams(method=0, rate_mx_per_hour=0.0)).to_c()
                                               for p in params])
        self._check(self.lib.sft_set_rfe(self.h, arr))

    def step(self, t_target, max_steps=0):
        n = C.c_int32(0)
        self._check(self.lib.sft_step(self.h, float(t_target), int(max_steps), C.byref(n)))
        return n.value

    def assimilate(self, obs, mu, per_realization, params):
        """per_realization: False/0 = one shared map, True/1 = one map per
        realization, 2 = one map per grid shape (shape order)."""
        if isinstance(params, AssimParams):
            params = [params] * self.n_real
        po, do, ko = _ptr(obs)
        pm, dm, km = _ptr(mu)
        if do != dm:
            raise ValueError("obs and mu must both be on the host or both on the device")
        arr = (sft_assim_params * self.n_real)(*[p.to_c() for p in params])
        mode = int(per_realization) if not isinstance(per_realization, bool) else (1 if per_realization else 0)
        self._check(self.lib.sft_assimilate(self.h, C.c_void_p(po), C.c_void_p(pm), mode, do, arr))
        del ko, km

    def balance_flux(self):
        self._check(self.lib.sft_balance_flux(self.h))

    def diagnostics(self, lat_cut_deg=60.0):
        out = (sft_diag * self.n_real)()
        self._check(self.lib.sft_flux_diagnostics(self.h, float(lat_cut_deg), out))
        return [{f[0]: getattr(d, f[0]) for f in sft_diag._fields_} for d in out]

    def stats(self):
        s = sft_stats()
        self._check(self.lib.sft_get_stats(self.h, C.byref(s)))
        return {f[0]: getattr(s, f[0]) for f in sft_stats._fields_}

    def reset_stats(self):
        self._check(self.lib.sft_reset_stats(self.h))

    def set_profiling(self, on):
        self._check(self.lib.sft_set_profiling(self.h, 1 if on else 0))

    def set_graphs(self, on):
        self._check(self.lib.sft_set_graphs(self.h, 1 if on else 0))

    def set_fusion(self, stages_per_pass):
        self._check(self.lib.sft_set_fusion(self.h, int(stages_per_pass)))

    def get_fusion(self):
        return self.lib.sft_get_fusion(self.h)

    def set_tile_rows(self, shape_id, rows):
        self._check(self.lib.sft_set_tile_rows(self.h, shape_id, rows))

    def get_tile_rows(self, shape_id):
        return self.lib.sft_get_tile_rows(self.h, shape_id)

    def set_band_rows(self, shape_id, rows):
        self._check(self.lib.sft_set_band_rows(self.h, shape_id, rows))

    def get_band_rows(self, shape_id):
        return self.lib.sft_get_band_rows(self.h, shape_id)

    def wave_size(self):
        return self.lib.sft_wave_size(self.h)

    def step_plan(self, r, dt):
        a, b, s = C.c_double(), C.c_double(), C.c_int32()
        self._check(self.lib.sft_step_plan(self.h, r, float(dt), C.byref(a), C.byref(b), C.byref(s)))
        return a.value, b.value, s.value


def flux_diagnostics_noalloc(br, lat_cut_deg=60.0, stream=None):
    """sft_flux_diagnostics_noalloc on a contiguous CUDA tensor [ntheta][nphi]
    (float32 or float64).  Allocates no device memory.  stream: a torch
    stream or raw handle; None = torch's current stream on br's device (the
    one a map written by torch was produced on)."""
    lib = load()
    import torch
    if not (isinstance(br, torch.Tensor) and br.is_cuda and br.is_contiguous() and br.dim() == 2):
        raise TypeError("expected a contiguous 2-D CUDA tensor")
    prec = {torch.float32: SFT_FP32, torch.float64: SFT_FP64}[br.dtype]
    if stream is None:
        stream = torch.cuda.current_stream(br.device)
    s = stream if isinstance(stream, int) else stream.cuda_stream
    out = sft_diag()
    st = lib.sft_flux_diagnostics_noalloc(C.c_void_p(br.data_ptr()), br.shape[0], br.shape[1], prec,
                                          float(lat_cut_deg), s, C.byref(out))
    if st != SFT_OK:
        raise SFTError(st, lib.sft_last_error(None).decode())
    return {f[0]: getattr(out, f[0]) for f in sft_diag._fields_}


__all__ = ["flux_diagnostics_noalloc", "Grid", "FlowParams", "AssimParams", "SFTError", "load", "header_functions",
           "LIB_PATH", "sft_flow_params", "sft_assim_params", "sft_diag", "sft_stats"]
del fields
