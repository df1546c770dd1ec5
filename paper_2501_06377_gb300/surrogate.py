"""Thin ctypes binding of the learned surrogate (include/sfs.h).

Marshalling only: the network's forward and backward passes, the optimizer
and the error reductions run in the CUDA kernels of libsft.so.  Maps and
parameters are CUDA torch tensors (float32, contiguous):
x, y [n, 256, 512] (Gauss), p [n, 5] = (o0, o2, o4 deg/day, U m/s, eta km^2/s).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .sft import SFT_OK, SFTError, load

H, W = 256, 512


class sfs_config(C.Structure):
    _fields_ = [("channels", C.c_int32), ("modes", C.c_int32), ("blocks", C.c_int32),
                ("max_batch", C.c_int32), ("seed", C.c_uint64)]


_SIGS = {
    "sfs_create": (C.c_int, [C.POINTER(sfs_config), C.c_void_p, C.POINTER(C.c_void_p)]),
    "sfs_destroy": (C.c_int, [C.c_void_p]),
    "sfs_num_params": (C.c_int64, [C.c_void_p]),
    "sfs_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sfs_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sfs_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sfs_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                C.POINTER(C.c_float), C.c_void_p]),
    "sfs_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                 C.c_double, C.c_double, C.POINTER(C.c_float)]),
    "sfs_rel_l2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sfs_flux": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sfs_set_sm_budget": (C.c_int, [C.c_void_p, C.c_int32]),
    "sfs_debug_gemm": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                 C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                 C.c_void_p, C.c_int64, C.c_int64, C.c_float, C.c_float, C.c_void_p, C.c_int32,
                                 C.c_int32]),
    "sfs_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                               C.POINTER(C.c_int64)]),
}

_bound = False


def _lib():
    global _bound
    lib = load()
    if not _bound:
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return lib


def _dev(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Surrogate:
    """One network with its optimizer state and work buffers."""

    def __init__(self, channels=64, modes=48, blocks=4, max_batch=32, seed=0, stream=None):
        self.lib = _lib()
        cfg = sfs_config(channels, modes, blocks, max_batch, seed)
        h = C.c_void_p()
        s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        st = self.lib.sfs_create(C.byref(cfg), s, C.byref(h))
        if st != SFT_OK:
            raise SFTError(st, self.lib.sft_last_error(None).decode())
        self.h = h
        self.channels, self.modes, self.blocks, self.max_batch = channels, modes, blocks, max_batch

    def _check(self, st):
        if st != SFT_OK:
            raise SFTError(st, self.lib.sft_last_error(None).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(self.lib.sfs_num_params(self.h))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.num_params()
        self._check(self.lib.sfs_set_params(self.h, C.c_void_p(a.ctypes.data)))

    def get_params(self):
        a = np.empty(self.num_params(), dtype=np.float32)
        self._check(self.lib.sfs_get_params(self.h, C.c_void_p(a.ctypes.data)))
        return a

    def forward(self, x, p, out):
        self._check(self.lib.sfs_forward(self.h, _dev(x), _dev(p), x.shape[0], _dev(out)))
        return out

    def loss_grad(self, x, p, y):
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = C.c_float()
        self._check(self.lib.sfs_loss_grad(self.h, _dev(x), _dev(p), _dev(y), x.shape[0], C.byref(loss),
                                           C.c_void_p(g.ctypes.data)))
        return float(loss.value), g

    def train_step(self, x, p, y, lr, wd=1e-4, want_loss=False):
        loss = C.c_float()
        self._check(self.lib.sfs_train_step(self.h, _dev(x), _dev(p), _dev(y), x.shape[0], float(lr),
                                            float(wd), C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def rel_l2(self, a, b):
        """||a - b|| / ||b|| per map (one call, one synchronisation)."""
        n = a.shape[0]
        out = np.empty(n, dtype=np.float64)
        self._check(self.lib.sfs_rel_l2(self.h, _dev(a), _dev(b), n, C.c_void_p(out.ctypes.data)))
        return out

    def flux(self, maps):
        """(signed, unsigned) FP64 flux of each map (one call, one synchronisation)."""
        n = maps.shape[0]
        o = np.empty(2 * n, dtype=np.float64)
        self._check(self.lib.sfs_flux(self.h, _dev(maps), n, C.c_void_p(o.ctypes.data)))
        o = o.reshape(-1, 2)
        return o[:, 0].copy(), o[:, 1].copy()

    def set_sm_budget(self, n_sm):
        """SMs the fused forward may occupy (0: all)."""
        self._check(self.lib.sfs_set_sm_budget(self.h, int(n_sm)))

    def debug_gemm(self, M, N, K, A, a_mn, lda, sA, B, b_mn, ldb, sB, Cm, ldc, sC, alpha=1.0, beta=0.0,
                   bias=None, kchunk=0, batch=1):
        """One tensor-core product C = alpha A B + beta C + bias (test entry
        point; A, B float32 or bfloat16 CUDA tensors, Cm float32)."""
        import torch

        def ptr(t):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype in (torch.float32, torch.bfloat16)):
                raise TypeError("expected a float32 or bfloat16 CUDA tensor")
            return C.c_void_p(t.data_ptr()), 1 if t.dtype == torch.bfloat16 else 0

        pa, abf = ptr(A)
        pb, bbf = ptr(B)
        self._check(self.lib.sfs_debug_gemm(self.h, M, N, K, pa, abf, a_mn, lda, sA, pb, bbf, b_mn, ldb, sB,
                                            _dev(Cm), ldc, sC, float(alpha), float(beta),
                                            _dev(bias) if bias is not None else None, kchunk, batch))

    def counters(self):
        g, f, k = C.c_int64(), C.c_double(), C.c_int64()
        self._check(self.lib.sfs_counters(self.h, C.byref(g), C.byref(f), C.byref(k)))
        return {"gemm_launches": g.value, "gemm_flops": f.value, "kernel_launches": k.value}


def flat_from_reference(P, blocks):
    """Flatten a reference parameter dict in the order of include/sfs.h."""
    parts = [P["We"], P["be"], P["Wd"], P["bd"]]
    for l in range(blocks):
        parts += [P["w%d" % l], P["W1_%d" % l], P["b1_%d" % l], P["W2_%d" % l], P["b2_%d" % l]]
    return np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in parts]).astype(np.float32)


def unflatten_like(flat, P, blocks):
    """Inverse of flat_from_reference (for comparing gradients)."""
    out, o = {}, 0
    order = ["We", "be", "Wd", "bd"]
    for l in range(blocks):
        order += ["w%d" % l, "W1_%d" % l, "b1_%d" % l, "W2_%d" % l, "b2_%d" % l]
    for k in order:
        n = P[k].size
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(P[k].shape)
        o += n
    return out
