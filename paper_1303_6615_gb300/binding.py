"""ctypes binding of libarp.so (include/arp.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes through; all computation runs in the library's CUDA
kernels.  Tensors are torch complex128 tensors of shape (batch, 3, N/2+1)
(device tensors unless a function accepts host memory); the stream defaults to
torch's current CUDA stream.  There is no CPU fallback: if the library cannot
be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libarp.so")

ARP_OK, ARP_EINVAL, ARP_ENOMEM, ARP_ECUDA, ARP_ETIMEOUT, ARP_ENONFINITE = range(6)
ARP_FP64, ARP_FP32 = 0, 1
ARP_OPT_T0, ARP_OPT_F, ARP_OPT_PRECISION, ARP_OPT_KMAX, ARP_OPT_TOL = 1, 2, 3, 4, 5
ARP_OPT_CHAIN = 6
ARP_TF32X3, ARP_BF16X2, ARP_BF16X3 = 2, 3, 4
ARP_OPT_FINE_BLOCK = 7
ARP_OPT_FINE_SCHEME = 8
ARP_OPT_COARSE_SCHEME = 9
ARP_OPT_COARSE_GRID = 10
ARP_OPT_PIPELINE = 11
ARP_OPT_TEST_SKIP_ARRIVAL = 100
STATUS_NAMES = {0: "ARP_OK", 1: "ARP_EINVAL", 2: "ARP_ENOMEM", 3: "ARP_ECUDA", 4: "ARP_ETIMEOUT",
                5: "ARP_ENONFINITE"}

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "arp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
    "arp_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "arp_query_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "arp_fine_batch": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "arp_coarse_avg": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "arp_coarse_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "arp_set_initial": (ctypes.c_int, [_P, _P, _P]),
    "arp_parareal_iterate": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_double)]),
    "arp_parareal_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]),
    "arp_get_slices": (ctypes.c_int, [_P, _P, _P]),
    "arp_destroy": (ctypes.c_int, [_P]),
    "arp_last_error": (ctypes.c_char_p, [_P]),
    "arp_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "arp_pipeline_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "arp_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "arp_gemm_check": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "arp_chain_exchange_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_uint)]),
    "arp_coarse_avg_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _P,
                                             _P, ctypes.c_int, _P]),
    "arp_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int]),
    "arp_batch_iterate": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "arp_batch_destroy": (ctypes.c_int, [_P]),
    "arp_batch_reset": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.c_int]),
    "arp_batch_last_error": (ctypes.c_char_p, [_P]),
}

_lib: Optional[ctypes.CDLL] = None


class ArpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libarp.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_1303_6615_gb300.build`)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(ctx, status: int):
    if status != ARP_OK:
        msg = load_library().arp_last_error(ctx)
        raise ArpError(status, msg.decode() if msg else "")


def _states(t, name: str, H: int):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a complex128 tensor")
    if t.dim() != 3 or t.shape[1] != 3 or t.shape[2] != H or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (batch, 3, {H}) tensor")
    return t.shape[0]


def arp_create(N: int, eps: float, nu: float, slices: int, dT: float, dt: float, M: int) -> int:
    lib = load_library()
    h = _P()
    st = lib.arp_create(ctypes.byref(h), N, eps, nu, slices, dT, dt, M)
    _check(None, st)
    return h.value


def arp_set_option(ctx: int, key: int, value: float) -> None:
    _check(ctx, load_library().arp_set_option(ctx, key, float(value)))


def arp_query_bytes(N: int, slices: int, M: int, precision: int) -> int:
    return load_library().arp_query_bytes(N, slices, M, precision)


def arp_info(ctx: int) -> dict:
    out = (ctypes.c_int * 9)()
    _check(ctx, load_library().arp_info(ctx, out))
    keys = ("N", "H", "K", "slices", "M", "steps", "level", "precision", "fine_schedule")
    return dict(zip(keys, list(out)))


def arp_alu_peak(precision: int, stream=None) -> float:
    """Measured plain-ALU peak (TFLOP/s) of the current device for ARP_FP32 or ARP_FP64."""
    t = ctypes.c_double(0.0)
    st = load_library().arp_alu_peak(precision, ctypes.byref(t), _stream(stream))
    if st != ARP_OK:
        raise ArpError(st, "arp_alu_peak failed")
    return t.value


def arp_chain_exchange_bytes(N: int, cluster: int, rank: int, precision: int) -> tuple[int, int]:
    """(red, ws): the bytes CTA `rank` of the chain's cluster expects per time average (host arithmetic)."""
    red, ws = ctypes.c_uint(0), ctypes.c_uint(0)
    st = load_library().arp_chain_exchange_bytes(N, cluster, rank, precision, ctypes.byref(red), ctypes.byref(ws))
    if st != ARP_OK:
        raise ArpError(st, "arp_chain_exchange_bytes failed")
    return red.value, ws.value


def arp_gemm_check(precision: int, A, B, C, stream=None) -> None:
    """C[j][i] = sum_k A[i][k] B[j][k] on the split-precision tensor-core kernel;
    A (m, k), B (n, k), C (n, m): contiguous float32 device tensors."""
    m, k = A.shape
    n = B.shape[0]
    st = load_library().arp_gemm_check(precision, m, n, k, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                       _stream(stream))
    if st != ARP_OK:
        raise ArpError(st, "arp_gemm_check failed")


def arp_pipeline_info(ctx: int) -> dict:
    out = (ctypes.c_int * 6)()
    _check(ctx, load_library().arp_pipeline_info(ctx, out))
    keys = ("pipelined", "chain_sms", "fine_sms", "chunk", "cluster", "refused")
    return dict(zip(keys, list(out)))


def _batch_call(fn_name: str, ctx: int, U_in, U_out, stream=None) -> None:
    H = arp_info(ctx)["H"]
    b = _states(U_in, "U_in", H)
    b2 = _states(U_out, "U_out", H)
    if b != b2:
        raise ValueError("U_in and U_out batch sizes differ")
    if b and (not U_in.is_cuda or not U_out.is_cuda):
        raise ValueError("U_in and U_out must be device tensors")
    fn = getattr(load_library(), fn_name)
    _check(ctx, fn(ctx, U_in.data_ptr() or None, U_out.data_ptr() or None, int(b), _stream(stream)))


def arp_fine_batch(ctx: int, U_in, U_out, stream=None) -> None:
    _batch_call("arp_fine_batch", ctx, U_in, U_out, stream)


def arp_coarse_avg(ctx: int, U_in, Nbar_out, stream=None) -> None:
    _batch_call("arp_coarse_avg", ctx, U_in, Nbar_out, stream)


def arp_coarse_step(ctx: int, U_in, U_out, stream=None) -> None:
    _batch_call("arp_coarse_step", ctx, U_in, U_out, stream)


def arp_coarse_avg_static(N: int, eps: float, dT: float, M: int, U_in, Nbar_out, stream=None) -> None:
    """Time average without a context or any device allocation (see include/arp.h)."""
    H = N // 2 + 1
    b = _states(U_in, "U_in", H)
    if _states(Nbar_out, "Nbar_out", H) != b:
        raise ValueError("U_in and Nbar_out batch sizes differ")
    if b and (not U_in.is_cuda or not Nbar_out.is_cuda):
        raise ValueError("U_in and Nbar_out must be device tensors")
    st = load_library().arp_coarse_avg_static(N, eps, dT, M, U_in.data_ptr() or None,
                                              Nbar_out.data_ptr() or None, int(b), _stream(stream))
    if st != ARP_OK:
        raise ArpError(st, "arp_coarse_avg_static failed")


def arp_set_initial(ctx: int, u0, stream=None) -> None:
    """u0: complex128 tensor (3, H) or (1, 3, H), host or device."""
    H = arp_info(ctx)["H"]
    t = u0.reshape(1, 3, H) if u0.dim() == 2 else u0
    _states(t, "u0", H)
    _check(ctx, load_library().arp_set_initial(ctx, t.data_ptr(), _stream(stream)))


def arp_parareal_iterate(ctx: int, stream=None) -> tuple[int, float]:
    k = ctypes.c_int(0)
    ch = ctypes.c_double(0.0)
    _check(ctx, load_library().arp_parareal_iterate(ctx, _stream(stream), ctypes.byref(k), ctypes.byref(ch)))
    return k.value, ch.value


def arp_parareal_solve(ctx: int, stream=None) -> tuple[int, float]:
    k = ctypes.c_int(0)
    ch = ctypes.c_double(0.0)
    _check(ctx, load_library().arp_parareal_solve(ctx, _stream(stream), ctypes.byref(k), ctypes.byref(ch)))
    return k.value, ch.value


def arp_get_slices(ctx: int, U, stream=None) -> None:
    """U: complex128 tensor (slices+1, 3, H), host or device."""
    info = arp_info(ctx)
    b = _states(U, "U", info["H"])
    if b != info["slices"] + 1:
        raise ValueError("U must hold slices+1 states")
    _check(ctx, load_library().arp_get_slices(ctx, U.data_ptr(), _stream(stream)))


def arp_destroy(ctx: int) -> None:
    if ctx:
        _check(None, load_library().arp_destroy(ctx))


def arp_last_error(ctx: Optional[int]) -> str:
    msg = load_library().arp_last_error(ctx)
    return msg.decode() if msg else ""


def arp_batch_create(ctxs, capacity: Optional[int] = None) -> int:
    """A batch of the contexts `ctxs`; ctxs=None with `capacity` gives an empty batch."""
    lib = load_library()
    h = _P()
    if ctxs is None:
        st = lib.arp_batch_create(ctypes.byref(h), None, int(capacity))
    else:
        arr = (_P * len(ctxs))(*ctxs)
        st = lib.arp_batch_create(ctypes.byref(h), arr, len(ctxs))
    if st != ARP_OK:
        raise ArpError(st, "arp_batch_create failed")
    return h.value


def arp_batch_iterate(batch: int, count: int, stream=None) -> tuple[list, list]:
    """One level for every context of the batch; returns (levels, changes)."""
    lib = load_library()
    lv = (ctypes.c_int * count)()
    ch = (ctypes.c_double * count)()
    st = lib.arp_batch_iterate(batch, _stream(stream), lv, ch)
    if st != ARP_OK:
        msg = lib.arp_batch_last_error(batch)
        raise ArpError(st, msg.decode() if msg else "")
    return list(lv), list(ch)


def arp_batch_reset(batch: int, ctxs) -> None:
    lib = load_library()
    arr = (_P * max(1, len(ctxs)))(*ctxs)
    st = lib.arp_batch_reset(batch, arr, len(ctxs))
    if st != ARP_OK:
        raise ArpError(st, arp_batch_last_error(batch))


def arp_batch_destroy(batch: int) -> None:
    if batch:
        load_library().arp_batch_destroy(batch)


def arp_batch_last_error(batch: int) -> str:
    msg = load_library().arp_batch_last_error(batch)
    return msg.decode() if msg else ""


class Solver:
    """Owning wrapper around one context (closes it on `close()` / exit)."""

    def __init__(self, N: int, eps: float, nu: float, slices: int, dT: float, dt: float, M: int,
                 precision: int = ARP_FP64, T0: Optional[float] = None, F: Optional[float] = None):
        self.ctx = arp_create(N, eps, nu, slices, dT, dt, M)
        try:
            if precision != ARP_FP64:
                arp_set_option(self.ctx, ARP_OPT_PRECISION, precision)
            if T0 is not None:
                arp_set_option(self.ctx, ARP_OPT_T0, T0)
            if F is not None:
                arp_set_option(self.ctx, ARP_OPT_F, F)
        except Exception:
            arp_destroy(self.ctx)
            raise
        self.info = arp_info(self.ctx)

    def close(self):
        if self.ctx:
            arp_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
