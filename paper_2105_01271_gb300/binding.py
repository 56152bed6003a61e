"""Thin ctypes binding of the C ABI in include/lrs.h.

Argument marshalling only: every step of the path runs in liblrs.so.  The
functions take torch CUDA tensors (or raw integer device pointers) plus the
sizes of the C signatures, and raise LrsError on a non-OK status (except
LRS_ERANK, which is returned, since the outputs are still valid at rank r).
There is no CPU fallback: loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LRS_OK, LRS_EINVAL, LRS_ENOMEM, LRS_ECUDA, LRS_ERANK, LRS_ETIMEOUT = range(6)
LRS_F64, LRS_F32, LRS_BF16 = 0, 1, 2
LRS_INJECT, LRS_FULLWEIGHT, LRS_BLOCKAVG = 0, 1, 2
LRS_PREC_FP64, LRS_PREC_FP32, LRS_PREC_SPLIT_BF16, LRS_PREC_BF16X3 = 0, 1, 2, 3
LRS_FACTOR_GRAM, LRS_FACTOR_R = 0, 1

KIND = {"inject": LRS_INJECT, "fullweight": LRS_FULLWEIGHT, "blockavg": LRS_BLOCKAVG}
DTYPE = {"f64": LRS_F64, "f32": LRS_F32, "bf16": LRS_BF16}
STATUS = {0: "LRS_OK", 1: "LRS_EINVAL", 2: "LRS_ENOMEM", 3: "LRS_ECUDA", 4: "LRS_ERANK",
          5: "LRS_ETIMEOUT"}


class LrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lrs_grid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("kind", C.c_int32), ("N", C.c_int64 * 3), ("s", C.c_int32 * 3)]


class lrs_batch_item(C.Structure):
    """Mirror of include/lrs.h's lrs_batch_item (one decomposition of a batch)."""
    _fields_ = [("A", C.c_void_p), ("dtype", C.c_int32), ("m", C.c_int64), ("lda", C.c_int64),
                ("sketch", lrs_grid), ("gram", lrs_grid),
                ("q", C.c_int32), ("k", C.c_int32), ("prec", C.c_int32), ("rtol", C.c_double),
                ("do_svd", C.c_int32), ("do_id", C.c_int32),
                ("U", C.c_void_p), ("ldu", C.c_int64), ("S", C.c_void_p), ("V", C.c_void_p),
                ("ldv", C.c_int64), ("J", C.c_void_p), ("P", C.c_void_p), ("ldp", C.c_int64),
                ("r", C.c_int64), ("err_svd", C.c_double), ("err_id", C.c_double), ("status", C.c_int32),
                ("launches", C.c_int64), ("error", C.c_char * 120)]


def make_grid(N, s, kind) -> lrs_grid:
    """lrs_grid from per-axis sizes (x first), factors and stencil name/code."""
    g = lrs_grid()
    g.ndim = len(N)
    g.kind = KIND[kind] if isinstance(kind, str) else int(kind)
    for d in range(3):
        g.N[d] = int(N[d]) if d < len(N) else 1
        g.s[d] = int(s[d]) if d < len(s) else 1
    return g


def grid_of(spec) -> lrs_grid:
    """lrs_grid from any object with N, s and kind attributes (e.g. synth.GridSpec)."""
    return make_grid(spec.N, spec.s, spec.kind)


_SIG = {
    "lrs_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "lrs_destroy": (None, [C.c_void_p]),
    "lrs_last_error": (C.c_char_p, [C.c_void_p]),
    "lrs_version": (C.c_char_p, []),
    "lrs_launch_count": (C.c_int64, [C.c_void_p]),
    "lrs_set_kernel_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "lrs_last_kernel_ms": (C.c_double, [C.c_void_p]),
    "lrs_set_workspace_limit": (C.c_int, [C.c_void_p, C.c_size_t]),
    "lrs_fp64_peak": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    "lrs_selftest_barrier_timeout": (C.c_int, [C.c_void_p, C.c_int64]),
    "lrs_sketch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64,
                             C.POINTER(lrs_grid), C.c_void_p, C.c_int64]),
    "lrs_power_pass": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64,
                                 C.POINTER(lrs_grid), C.POINTER(lrs_grid), C.c_int32, C.c_int32,
                                 C.c_double, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_int64, C.POINTER(C.c_int64)]),
    "lrs_power_pass2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64,
                                  C.POINTER(lrs_grid), C.POINTER(lrs_grid), C.c_int32, C.c_double,
                                  C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_int64), C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "lrs_touch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.POINTER(lrs_grid),
                            C.POINTER(lrs_grid), C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "lrs_power_pass_from": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                      C.c_int64, C.c_int64, C.c_int32, C.c_double, C.c_int32, C.c_void_p,
                                      C.c_int64, C.POINTER(C.c_int64), C.c_void_p, C.c_int64,
                                      C.POINTER(C.c_int64)]),
    "lrs_apass_slab": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                                 C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]),
    "lrs_slab_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                  C.c_void_p, C.c_int64]),
    "lrs_svd_from_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                      C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_int64, C.POINTER(C.c_double)]),
    "lrs_range_find": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                 C.c_double, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "lrs_range_find_diag": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                      C.c_double, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "lrs_svd_k": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                            C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                            C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_id_k": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                           C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_id_k_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_gemm_tn": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int32,
                              C.c_int64, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int32,
                              C.c_int32, C.c_int64, C.c_int32]),
    "lrs_batch_run": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.c_int32]),
    "lrs_batch_autotune": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.c_int32,
                                     C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "lrs_batch_release": (C.c_int, [C.c_int]),
    "lrs_batch_graph_create": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_void_p)]),
    "lrs_batch_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "lrs_batch_graph_destroy": (None, [C.c_void_p]),
    "lrs_range_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                                  C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_sketch_svd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_double,
                                 C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "lrs_spc_lift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                               C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                               C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_int32,
                               C.c_void_p, C.c_int64]),
    "lrs_spc_err": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                              C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_double), C.c_int32,
                              C.POINTER(C.c_double)]),
    "lrs_spc_stream_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                                        C.c_int32, C.POINTER(C.c_void_p)]),
    "lrs_spc_stream_push": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32]),
    "lrs_spc_stream_svd": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_spc_stream_id": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_int64, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lrs_spc_stream_err": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double)]),
    "lrs_spc_stream_cpwr": (C.c_int, [C.c_void_p, C.POINTER(lrs_grid), C.c_int32]),
    "lrs_spc_stream_cpwr_svd": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                          C.POINTER(C.c_int64)]),
    "lrs_spc_stream_cpwr_id": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_int64, C.POINTER(C.c_double)]),
    "lrs_spc_stream_sketch": (C.c_void_p, [C.c_void_p]),
    "lrs_spc_stream_destroy": (None, [C.c_void_p]),
    "lrs_spc_stream_reset": (C.c_int, [C.c_void_p]),
    "lrs_mlp_param_count": (C.c_int64, []),
    "lrs_mlp_init_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lrs_mlp_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                   C.c_void_p]),
    "lrs_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "lrs_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_void_p]),
    "lrs_mlp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int64, C.c_float]),
}

EXPORTS = tuple(_SIG)

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """dlopen liblrs.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"liblrs.so not found at {path}; run paper_2105_01271_gb300/build.py")
    lib = C.CDLL(path)
    for name, (res, args) in _SIG.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x.ctypes.data)              # a numpy array in host memory


class Context:
    """One lrs_ctx bound to a device and a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        h = C.c_void_p()
        sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        st = self.lib.lrs_create(C.byref(h), int(device), C.c_void_p(sp))
        if st != LRS_OK:
            raise LrsError(st, "lrs_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow_rank=False):
        if st == LRS_OK or (allow_rank and st == LRS_ERANK):
            return st
        raise LrsError(st, self.lib.lrs_last_error(self.h).decode())

    @property
    def launches(self) -> int:
        return int(self.lib.lrs_launch_count(self.h))

    def set_kernel_timing(self, on: bool):
        return self._check(self.lib.lrs_set_kernel_timing(self.h, 1 if on else 0))

    def last_kernel_ms(self) -> float:
        return float(self.lib.lrs_last_kernel_ms(self.h))

    def fp64_peak(self, iters: int = 4096) -> float:
        """Measured FP64 FMA throughput of the device, TFLOP/s (lrs_fp64_peak)."""
        t = C.c_double(0.0)
        self._check(self.lib.lrs_fp64_peak(self.h, int(iters), C.byref(t)))
        return t.value

    def set_workspace_limit(self, nbytes: int):
        return self._check(self.lib.lrs_set_workspace_limit(self.h, int(nbytes)))

    def selftest_barrier_timeout(self, spin_limit: int) -> int:
        """Status of the forced barrier timeout (LRS_ETIMEOUT expected); does not raise."""
        return int(self.lib.lrs_selftest_barrier_timeout(self.h, int(spin_limit)))

    # --- the C ABI, one wrapper per entry point -----------------------------
    def sketch(self, A, dtype, m, lda, grid: lrs_grid, Y, ldy):
        return self._check(self.lib.lrs_sketch(self.h, _ptr(A), dtype, m, lda, C.byref(grid),
                                               _ptr(Y), ldy))

    def power_pass(self, A, dtype, m, lda, sketch: lrs_grid, gram, q, reorth, rtol, prec,
                   Y, ldy, G, ldg) -> int:
        gc = C.c_int64(0)
        gp = C.byref(gram) if gram is not None else None
        self._check(self.lib.lrs_power_pass(self.h, _ptr(A), dtype, m, lda, C.byref(sketch), gp,
                                            q, reorth, rtol, prec, _ptr(Y), ldy, _ptr(G), ldg,
                                            C.byref(gc)))
        return gc.value

    def power_pass2(self, A, dtype, m, lda, sketch: lrs_grid, gram, q, rtol, prec,
                    Y, ldy, G0, ldg0, G, ldg):
        """Returns (columns of G0, columns of G)."""
        gc = C.c_int64(0)
        g0 = C.c_int64(0)
        gp = C.byref(gram) if gram is not None else None
        self._check(self.lib.lrs_power_pass2(self.h, _ptr(A), dtype, m, lda, C.byref(sketch), gp,
                                             q, rtol, prec, _ptr(Y), ldy, _ptr(G0), ldg0, C.byref(g0),
                                             _ptr(G), ldg, C.byref(gc)))
        return g0.value, gc.value

    def touch(self, A, dtype, m, lda, sketch: lrs_grid, gram, prec, Y, ldy, W, ldw):
        gp = C.byref(gram) if gram is not None else None
        return self._check(self.lib.lrs_touch(self.h, _ptr(A), dtype, m, lda, C.byref(sketch), gp, prec,
                                              _ptr(Y), ldy, _ptr(W), ldw))

    def power_pass_from(self, Y, ldy, W, ldw, m, l, nI, q, rtol, prec, G0, ldg0, G, ldg):
        """Returns (columns of G0, columns of G)."""
        gc = C.c_int64(0)
        g0 = C.c_int64(0)
        self._check(self.lib.lrs_power_pass_from(self.h, _ptr(Y), ldy, _ptr(W), ldw, m, l, nI, q, rtol, prec,
                                                 _ptr(G0), ldg0, C.byref(g0), _ptr(G), ldg, C.byref(gc)))
        return g0.value, gc.value

    def apass_slab(self, A, dtype, m, n, lda, Q, ldq, r, prec, B, fro2):
        return self._check(self.lib.lrs_apass_slab(self.h, _ptr(A), dtype, m, n, lda, _ptr(Q), ldq, r, prec,
                                                   _ptr(B), _ptr(fro2)))

    def slab_factor(self, B, r, n, prec, mode, F, ldf):
        return self._check(self.lib.lrs_slab_factor(self.h, _ptr(B), r, n, prec, mode, _ptr(F), ldf))

    def svd_from_factor(self, F, ldf, nf, mode, Q, ldq, m, r, k, prec, B, n, fro2, U, ldu, S, V, ldv):
        """Returns (err_est, status); LRS_ERANK is returned, not raised."""
        err = C.c_double(0.0)
        st = self._check(self.lib.lrs_svd_from_factor(self.h, _ptr(F), ldf, nf, mode, _ptr(Q), ldq, m, r, k, prec,
                                                      _ptr(B), n, _ptr(fro2), _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                                                      C.byref(err)), allow_rank=True)
        return err.value, st

    def range_find(self, G, m, l, ldg, rtol, Q, ldq) -> int:
        r = C.c_int64(0)
        self._check(self.lib.lrs_range_find(self.h, _ptr(G), m, l, ldg, rtol, _ptr(Q), ldq,
                                            C.byref(r)))
        return r.value

    def range_find_diag(self, G, m, l, ldg, rtol, Q, ldq, rdiag) -> int:
        r = C.c_int64(0)
        self._check(self.lib.lrs_range_find_diag(self.h, _ptr(G), m, l, ldg, rtol, _ptr(Q), ldq,
                                                 C.byref(r), _ptr(rdiag)))
        return r.value

    def svd_k(self, A, dtype, m, n, lda, Q, ldq, r, k, prec, U, ldu, S, V, ldv):
        err = C.c_double(0.0)
        st = self._check(self.lib.lrs_svd_k(self.h, _ptr(A), dtype, m, n, lda, _ptr(Q), ldq, r, k,
                                            prec, _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                                            C.byref(err)), allow_rank=True)
        return err.value, st

    def id_k(self, Ysk, m, l, ldy, k, J, P, ldp):
        err = C.c_double(0.0)
        st = self._check(self.lib.lrs_id_k(self.h, _ptr(Ysk), m, l, ldy, k, _ptr(J), _ptr(P), ldp,
                                           C.byref(err)), allow_rank=True)
        return err.value, st

    def id_k_static(self, Ysk, m, l, ldy, k, J, P, ldp):
        err = C.c_double(0.0)
        st = self._check(self.lib.lrs_id_k_static(self.h, _ptr(Ysk), m, l, ldy, k, _ptr(J), _ptr(P), ldp,
                                                  C.byref(err)), allow_rank=True)
        return err.value, st

    def range_error(self, A, dtype, m, n, lda, Q, ldq, r) -> float:
        err = C.c_double(0.0)
        self._check(self.lib.lrs_range_error(self.h, _ptr(A), dtype, m, n, lda, _ptr(Q), ldq, r, C.byref(err)))
        return err.value

    def sketch_svd(self, Y, m, l, ldy, rtol, Q, ldq, r, U, ldu, S, V, ldv) -> int:
        rank = C.c_int64(0)
        self._check(self.lib.lrs_sketch_svd(self.h, _ptr(Y), m, l, ldy, rtol, _ptr(Q), ldq, r, _ptr(U), ldu,
                                            _ptr(S), _ptr(V), ldv, C.byref(rank)))
        return rank.value

    def spc_lift(self, A, dtype, m, n, lda, Y, l, ldy, U, ldu, S, V, ldv, r, J, k, prec, Sf, ldsf):
        return self._check(self.lib.lrs_spc_lift(self.h, _ptr(A), dtype, m, n, lda, _ptr(Y), l, ldy, _ptr(U), ldu,
                                                 _ptr(S), _ptr(V), ldv, r, _ptr(J), k, prec, _ptr(Sf), ldsf))

    def spc_err(self, A, dtype, m, n, lda, Y, l, ldy, c, taus) -> list:
        nt = len(taus)
        t = (C.c_double * nt)(*[float(x) for x in taus])
        out = (C.c_double * nt)()
        self._check(self.lib.lrs_spc_err(self.h, _ptr(A), dtype, m, n, lda, _ptr(Y), l, ldy, c, t, nt, out))
        return list(out)

    def mlp_init_bf16(self, params, wbf16):
        return self._check(self.lib.lrs_mlp_init_bf16(self.h, _ptr(params), _ptr(wbf16)))

    def mlp_features(self, rdiag, ns, r, l, N, m, x):
        return self._check(self.lib.lrs_mlp_features(self.h, _ptr(rdiag), ns, r, l, N, m, _ptr(x)))

    def mlp_forward(self, params, wbf16, X, B, logits):
        return self._check(self.lib.lrs_mlp_forward(self.h, _ptr(params), _ptr(wbf16), _ptr(X), B, _ptr(logits)))

    def mlp_loss_grad(self, params, wbf16, X, y, B, grad, loss):
        return self._check(self.lib.lrs_mlp_loss_grad(self.h, _ptr(params), _ptr(wbf16), _ptr(X), _ptr(y), B,
                                                      _ptr(grad), _ptr(loss)))

    def mlp_adam(self, params, wbf16, grad, m1, m2, step, lr):
        return self._check(self.lib.lrs_mlp_adam(self.h, _ptr(params), _ptr(wbf16), _ptr(grad), _ptr(m1), _ptr(m2),
                                                 step, lr))

    def gemm_tn(self, M, N, K, X, x_dtype, ldx, A, a_dtype, lda, Cm, c_f64, c_trans, ldc, prec):
        return self._check(self.lib.lrs_gemm_tn(self.h, M, N, K, _ptr(X), x_dtype, ldx, _ptr(A),
                                                a_dtype, lda, _ptr(Cm), c_f64, c_trans, ldc, prec))


class SpcStream:
    """lrs_spc_stream: the single read of streamed snapshots (Algs. 3, 5, 6).
    Keep the Context alive while the stream exists."""

    def __init__(self, ctx: Context, dtype: int, m: int, sketch: lrs_grid, block_rows: int, err_c: int = 0,
                 prec: int = LRS_PREC_SPLIT_BF16):
        self.ctx = ctx
        self.lib = ctx.lib
        h = C.c_void_p()
        ctx._check(self.lib.lrs_spc_stream_create(ctx.h, dtype, m, C.byref(sketch), block_rows, err_c, prec,
                                                  C.byref(h)))
        self.h = h

    def push(self, rows, nrows: int, ld: int, on_device: bool):
        return self.ctx._check(self.lib.lrs_spc_stream_push(self.h, _ptr(rows), nrows, ld, 1 if on_device else 0))

    def svd(self, rtol, r, k, U, ldu, S, V, ldv) -> float:
        err = C.c_double(0.0)
        self.ctx._check(self.lib.lrs_spc_stream_svd(self.h, rtol, r, k, _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                                                    C.byref(err)))
        return err.value

    def id(self, rtol, r, k, J, P, ldp, Sf, ldsf) -> float:
        err = C.c_double(0.0)
        self.ctx._check(self.lib.lrs_spc_stream_id(self.h, rtol, r, k, _ptr(J), _ptr(P), ldp, _ptr(Sf), ldsf,
                                                   C.byref(err)))
        return err.value

    def err(self, taus) -> list:
        nt = len(taus)
        t = (C.c_double * nt)(*[float(x) for x in taus])
        out = (C.c_double * nt)()
        self.ctx._check(self.lib.lrs_spc_stream_err(self.h, t, nt, out))
        return list(out)

    def enable_cpwr(self, gram: lrs_grid, spc_too: bool = True):
        """lrs_spc_stream_cpwr: C-PWR's subsample and W^T A_f in the same read
        (spc_too = False: without the SPC finishers' H^T)."""
        return self.ctx._check(self.lib.lrs_spc_stream_cpwr(self.h, C.byref(gram), 1 if spc_too else 0))

    def cpwr_svd(self, q, rtol, k, U, ldu, S, V, ldv):
        """Returns (err_est, r, status); LRS_ERANK is returned, not raised."""
        err, r = C.c_double(0.0), C.c_int64(0)
        st = self.ctx._check(self.lib.lrs_spc_stream_cpwr_svd(self.h, q, rtol, k, _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                                                              C.byref(err), C.byref(r)), allow_rank=True)
        return err.value, r.value, st

    def cpwr_id(self, q, rtol, k, J, P, ldp) -> float:
        err = C.c_double(0.0)
        self.ctx._check(self.lib.lrs_spc_stream_cpwr_id(self.h, q, rtol, k, _ptr(J), _ptr(P), ldp, C.byref(err)))
        return err.value

    def sketch_ptr(self) -> int:
        return int(self.lib.lrs_spc_stream_sketch(self.h) or 0)

    def reset(self):
        return self.ctx._check(self.lib.lrs_spc_stream_reset(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrs_spc_stream_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def run_batch(items, device: int = 0, n_streams: int = 4) -> int:
    """lrs_batch_run over a ctypes array of lrs_batch_item (status per item in
    items[i].status); raises LrsError unless every item ended OK or ERANK."""
    lib = load_library()
    st = lib.lrs_batch_run(int(device), C.cast(items, C.c_void_p), len(items), int(n_streams))
    if st != LRS_OK:
        bad = [(i, it.status, it.error.decode(errors="replace")) for i, it in enumerate(items)
               if it.status not in (LRS_OK, LRS_ERANK)]
        raise LrsError(st, f"batch: {len(bad)} item(s) failed, first {bad[:3]}")
    return st


def autotune_batch(items, device: int = 0, candidates=(1, 2, 4, 8)):
    """lrs_batch_autotune: (best stream count, ms per sampled item)."""
    lib = load_library()
    cand = (C.c_int32 * len(candidates))(*candidates)
    best, ms = C.c_int32(0), C.c_double(0.0)
    st = lib.lrs_batch_autotune(int(device), C.cast(items, C.c_void_p), len(items), cand, len(candidates),
                                C.byref(best), C.byref(ms))
    if st != LRS_OK:
        bad = [(i, it.status, it.error.decode(errors="replace")) for i, it in enumerate(items)
               if it.status not in (LRS_OK, LRS_ERANK)]
        raise LrsError(st, f"batch autotune: {len(bad)} item(s) failed, first {bad[:3]}")
    return best.value, ms.value


class BatchGraph:
    """lrs_batch_graph: the batch captured as one CUDA graph (items with q = 0).
    Creating it runs the batch once (the results are written to the items);
    launch() replays the whole batch with one graph launch."""

    def __init__(self, items, device: int = 0, branches: int = 4):
        lib = load_library()
        self.lib = lib
        h = C.c_void_p()
        st = lib.lrs_batch_graph_create(int(device), C.cast(items, C.c_void_p), len(items), int(branches), C.byref(h))
        if st != LRS_OK:
            bad = [(i, it.status, it.error.decode(errors="replace")) for i, it in enumerate(items)
                   if it.status not in (LRS_OK, LRS_ERANK) or it.error[:1]]
            if not h.value:
                raise LrsError(st, f"batch graph: {bad[:3]}")
        self.h = h

    def launch(self, items) -> int:
        """Replays the batch; returns how many items were run again eagerly."""
        n = C.c_int64(0)
        st = self.lib.lrs_batch_graph_launch(self.h, C.cast(items, C.c_void_p), len(items), C.byref(n))
        if st != LRS_OK:
            bad = [(i, it.status, it.error.decode(errors="replace")) for i, it in enumerate(items)
                   if it.status not in (LRS_OK, LRS_ERANK)]
            raise LrsError(st, f"batch graph launch: {bad[:3]}")
        return n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrs_batch_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
