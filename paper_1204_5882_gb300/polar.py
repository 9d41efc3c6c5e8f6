"""Thin ctypes binding of the C ABI in ``include/polar.h``.

Argument marshalling only: every function forwards to the CUDA library with
the same name; device buffers are PyTorch tensors passed as raw pointers,
streams as ``torch.cuda.Stream.cuda_stream``.  There is no fallback: if the
library has not been built, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB_PATH

POLAR_OK, POLAR_EINVAL, POLAR_ENOMEM, POLAR_ECUDA = 0, -1, -2, -3
POLAR_ETIMEDOUT, POLAR_EBUSY, POLAR_ENOTFOUND, POLAR_PENDING = -4, -5, -6, 1
POLAR_ECANCELED, POLAR_EFAULT = -7, -8
POLAR_BSC, POLAR_BIAWGN = 0, 1
POLAR_F_MINSUM, POLAR_F_EXACT = 0, 1
POLAR_FP32, POLAR_FP16, POLAR_INT8 = 0, 1, 2

CHANNEL = {"bsc": POLAR_BSC, "biawgn": POLAR_BIAWGN}
FKIND = {"minsum": POLAR_F_MINSUM, "exact": POLAR_F_EXACT}
PREC = {"fp32": POLAR_FP32, "fp16": POLAR_FP16, "int8": POLAR_INT8}


class PolarError(RuntimeError):
    def __init__(self, fn, status):
        msg = f"{fn} failed: {status} ({_lib.polar_strerror(status).decode()})"
        extra = _lib.polar_last_error_string().decode()
        if status == POLAR_ECUDA and extra:
            msg += f": {extra}"
        super().__init__(msg)
        self.status = status


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int), ("max_inflight", C.c_int), ("max_queue", C.c_int),
                ("mem_budget", C.c_size_t), ("fkind", C.c_int), ("prec", C.c_int),
                ("threads", C.c_int), ("persistent", C.c_int), ("max_log2n", C.c_int)]


class Request(C.Structure):
    _fields_ = [("fs", C.c_void_p), ("nframes", C.c_int), ("llr", C.c_void_p),
                ("frozen_vals", C.c_void_p), ("xhat", C.c_void_p), ("uhat", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


class FrameDesc(C.Structure):
    _fields_ = [("fs", C.c_void_p), ("llr", C.c_void_p), ("frozen_vals", C.c_void_p),
                ("xhat", C.c_void_p), ("uhat", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    P, I, U32, U64, D, SZ = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double, C.c_size_t
    sig = {
        "polar_strerror": ([I], C.c_char_p),
        "polar_last_error_string": ([], C.c_char_p),
        "polar_config_set": ([C.c_char_p, C.c_long], I),
        "polar_config_get": ([C.c_char_p, C.POINTER(C.c_long)], I),
        "polar_kernel_launches": ([], U64),
        "polar_profile_read": ([C.c_char_p, C.POINTER(D), C.POINTER(U64), C.POINTER(D)], I),
        "polar_profile_reset": ([], None),
        "polar_build_frozen_set": ([U32, I, D, D, C.POINTER(P)], I),
        "polar_frozen_set_from_mask": ([U32, P, C.POINTER(P)], I),
        "polar_build_frozen_set_tv": ([U32, I, D, I, D, D, C.POINTER(P)], I),
        "polar_build_frozen_set_sum": ([U32, I, D, D, C.POINTER(P)], I),
        "polar_build_frozen_set_device": ([U32, I, D, D, D, P, C.POINTER(P)], I),
        "polar_frozen_set_query": ([P, C.POINTER(U32), C.POINTER(U64), P, C.POINTER(D)], I),
        "polar_frozen_set_free": ([P], None),
        "polar_llr_from_channel": ([I, D, P, I, P, SZ, P], I),
        "polar_encode": ([U32, I, P, P, P], I),
        "polar_reveal": ([P, I, P, P, P], I),
        "polar_sc_decode": ([P, P, P, P, P, I, I, P], I),
        "polar_sc_decode_many": ([P, I, P, P, P, P, I, I, P], I),
        "polar_sc_decode_batch": ([I, C.POINTER(FrameDesc), I, I, P], I),
        "polar_sc_decode_persistent": ([I, C.POINTER(FrameDesc), I, I, P], I),
        "polar_sc_decode_many_noalloc": ([P, I, P, P, P, P, I, I, P], I),
        "polar_autotune": ([P, I, P, P, P, I, I, P, C.POINTER(I), C.POINTER(I),
                            C.POINTER(D)], I),
        "polar_tune_save": ([C.c_char_p], I),
        "polar_tune_load": ([C.c_char_p], I),
        "polar_tune_clear": ([], None),
        "polar_frame_hash": ([U32, I, P, U64, P, P], I),
        "polar_key_rate": ([D, D, D, D, D], D),
        "polar_server_create": ([C.POINTER(ServerConfig), C.POINTER(P)], I),
        "polar_server_submit": ([P, C.POINTER(Request), C.POINTER(U64)], I),
        "polar_server_poll": ([P, U64, C.POINTER(Result)], I),
        "polar_server_wait": ([P, U64, D, C.POINTER(Result)], I),
        "polar_server_cancel": ([P, U64], I),
        "polar_debug_spoil_guard": ([P], I),
        "polar_frozen_set_upload": ([P, I], I),
        "polar_server_stats": ([P, C.POINTER(U64), C.POINTER(U64), C.POINTER(U64),
                                C.POINTER(SZ)], I),
        "polar_server_destroy": ([P], None),
        "polar_static_scratch_bytes": ([], SZ),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def _check(fn, rc):
    if rc != POLAR_OK:
        raise PolarError(fn, rc)
    return rc


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ config
def polar_config_set(key: str, value: int):
    _check("polar_config_set", _lib.polar_config_set(key.encode(), int(value)))


def polar_frozen_set_upload(fs, device=0):
    """Make the frozen set resident on `device` (mask and class tables)."""
    _check("polar_frozen_set_upload", _lib.polar_frozen_set_upload(fs.handle, int(device)))


def polar_debug_spoil_guard(stream=None):
    """Guard-mode self-test: spoil the trailing guard zone of the scratch
    that the last decode on `stream` used."""
    _check("polar_debug_spoil_guard", _lib.polar_debug_spoil_guard(_stream(stream)))


def polar_config_get(key: str) -> int:
    v = C.c_long()
    _check("polar_config_get", _lib.polar_config_get(key.encode(), C.byref(v)))
    return v.value


def polar_kernel_launches() -> int:
    return int(_lib.polar_kernel_launches())


def polar_profile_read(kind: str):
    """(total_ms, launches, algorithmic_bytes) recorded for one kernel kind."""
    ms, n, b = C.c_double(), C.c_uint64(), C.c_double()
    _check("polar_profile_read", _lib.polar_profile_read(kind.encode(), C.byref(ms), C.byref(n),
                                                         C.byref(b)))
    return ms.value, n.value, b.value


def polar_profile_reset():
    _lib.polar_profile_reset()


PROFILE_KINDS = ("llr", "stream_f", "stream_g", "subtree", "rate0", "chain", "persist",
                 "node")


# ------------------------------------------------------------------ frozen sets
class FrozenSet:
    """Owner of a library frozen-set object (freed on garbage collection)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)
        n, k, s = C.c_uint32(), C.c_uint64(), C.c_double()
        _check("polar_frozen_set_query", _lib.polar_frozen_set_query(
            self.handle, C.byref(n), C.byref(k), None, C.byref(s)))
        self.log2n, self.K, self.sum_pe = n.value, k.value, s.value
        self.N = 1 << self.log2n
        self.words = max(1, self.N // 32)

    def mask(self) -> np.ndarray:
        m = np.empty(self.words, dtype=np.uint32)
        _check("polar_frozen_set_query", _lib.polar_frozen_set_query(
            self.handle, None, None, m.ctypes.data_as(C.c_void_p), None))
        return m

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.polar_frozen_set_free(self.handle)
            self.handle = None


def polar_build_frozen_set_sum(log2n: int, channel: str, param: float,
                               sum_pe_max: float = 0.1) -> FrozenSet:
    """Bhattacharyya / GA set with K chosen by the sum rule (Sec. 3)."""
    h = C.c_void_p()
    _check("polar_build_frozen_set_sum", _lib.polar_build_frozen_set_sum(
        int(log2n), CHANNEL[channel], float(param), float(sum_pe_max), C.byref(h)))
    return FrozenSet(h.value)


def polar_build_frozen_set_device(log2n: int, channel: str, param: float, rate: float = 0.0,
                                  sum_pe_max: float = 0.1, stream=None) -> FrozenSet:
    """Bhattacharyya / GA set built on the GPU in double precision; K =
    floor(rate N), or with rate = 0 by the sum rule (Sec. 3)."""
    h = C.c_void_p()
    _check("polar_build_frozen_set_device", _lib.polar_build_frozen_set_device(
        int(log2n), CHANNEL[channel], float(param), float(rate), float(sum_pe_max),
        _stream(stream), C.byref(h)))
    return FrozenSet(h.value)


def polar_build_frozen_set_tv(log2n: int, channel: str, param: float, mu: int = 16,
                              rate: float = 0.0, sum_pe_max: float = 0.1) -> FrozenSet:
    """Degraded-channel construction; K = floor(rate N), or by the sum rule."""
    h = C.c_void_p()
    _check("polar_build_frozen_set_tv", _lib.polar_build_frozen_set_tv(
        int(log2n), CHANNEL[channel], float(param), int(mu), float(rate), float(sum_pe_max),
        C.byref(h)))
    return FrozenSet(h.value)


def polar_build_frozen_set(log2n: int, channel: str, param: float, rate: float) -> FrozenSet:
    h = C.c_void_p()
    _check("polar_build_frozen_set", _lib.polar_build_frozen_set(
        int(log2n), CHANNEL[channel], float(param), float(rate), C.byref(h)))
    return FrozenSet(h.value)


def polar_frozen_set_from_mask(log2n: int, mask_words) -> FrozenSet:
    m = np.ascontiguousarray(np.asarray(mask_words, dtype=np.uint32))
    h = C.c_void_p()
    _check("polar_frozen_set_from_mask", _lib.polar_frozen_set_from_mask(
        int(log2n), m.ctypes.data_as(C.c_void_p), C.byref(h)))
    return FrozenSet(h.value)


# ------------------------------------------------------------------ channel / Alice
def polar_llr_from_channel(channel: str, param: float, y, llr, stream=None):
    import torch
    bits = y.dtype in (torch.int32, torch.uint32)
    _check("polar_llr_from_channel", _lib.polar_llr_from_channel(
        CHANNEL[channel], float(param), _ptr(y), 1 if bits else 0, _ptr(llr), llr.numel(),
        _stream(stream)))


def polar_encode(log2n: int, nframes: int, inp, out, stream=None):
    _check("polar_encode", _lib.polar_encode(int(log2n), int(nframes), _ptr(inp), _ptr(out),
                                             _stream(stream)))


def polar_reveal(fs: FrozenSet, nframes: int, x, fval, stream=None):
    _check("polar_reveal", _lib.polar_reveal(fs.handle, int(nframes), _ptr(x), _ptr(fval),
                                             _stream(stream)))


# ------------------------------------------------------------------ decoding
def polar_sc_decode(fs: FrozenSet, llr, fval, xhat, uhat=None, fkind="minsum", prec="fp32",
                    stream=None):
    _check("polar_sc_decode", _lib.polar_sc_decode(
        fs.handle, _ptr(llr), _ptr(fval), _ptr(xhat), _ptr(uhat), FKIND[fkind], PREC[prec],
        _stream(stream)))


def polar_sc_decode_many(fs: FrozenSet, nframes: int, llr, fval, xhat, uhat=None,
                         fkind="minsum", prec="fp32", stream=None):
    _check("polar_sc_decode_many", _lib.polar_sc_decode_many(
        fs.handle, int(nframes), _ptr(llr), _ptr(fval), _ptr(xhat), _ptr(uhat), FKIND[fkind],
        PREC[prec], _stream(stream)))


def _frame_descs(frames):
    arr = (FrameDesc * len(frames))()
    for i, (fs, llr, fv, xh, uh) in enumerate(frames):
        arr[i] = FrameDesc(fs.handle.value, llr.data_ptr(), fv.data_ptr(), xh.data_ptr(),
                           uh.data_ptr() if uh is not None else None)
    return arr


def polar_sc_decode_batch(frames, fkind="minsum", prec="fp32", stream=None):
    """frames: list of (FrozenSet, llr, fval, xhat, uhat_or_None) tensors."""
    _check("polar_sc_decode_batch", _lib.polar_sc_decode_batch(
        len(frames), _frame_descs(frames), FKIND[fkind], PREC[prec], _stream(stream)))


def polar_sc_decode_persistent(frames, fkind="minsum", prec="fp32", stream=None):
    """One persistent launch over frames of any lengths and codes; frames as
    for polar_sc_decode_batch."""
    _check("polar_sc_decode_persistent", _lib.polar_sc_decode_persistent(
        len(frames), _frame_descs(frames), FKIND[fkind], PREC[prec], _stream(stream)))


def polar_sc_decode_many_noalloc(fs: FrozenSet, nframes: int, llr, fval, xhat, uhat=None,
                                 fkind="minsum", prec="fp32", stream=None):
    _check("polar_sc_decode_many_noalloc", _lib.polar_sc_decode_many_noalloc(
        fs.handle, int(nframes), _ptr(llr), _ptr(fval), _ptr(xhat), _ptr(uhat), FKIND[fkind],
        PREC[prec], _stream(stream)))


# ------------------------------------------------------------------ verification
def polar_frame_hash(log2n: int, nframes: int, words, key: int, out, stream=None):
    """Keyed hash of each packed frame into out (uint64 / int64 tensor)."""
    _check("polar_frame_hash", _lib.polar_frame_hash(
        int(log2n), int(nframes), _ptr(words), int(key) & (2 ** 64 - 1), _ptr(out),
        _stream(stream)))


def polar_key_rate(alpha: float, fer: float, beta: float, mutual_info: float,
                   eve_info: float) -> float:
    return _lib.polar_key_rate(float(alpha), float(fer), float(beta), float(mutual_info),
                               float(eve_info))


# ------------------------------------------------------------------ autotuning
def polar_autotune(fs: FrozenSet, nframes: int, llr, fval, xhat, fkind="minsum", prec="fp32",
                   stream=None):
    """(best_t, best_fuse, best_ms) for this batch shape; later decodes use it."""
    t, fu, ms = C.c_int(), C.c_int(), C.c_double()
    _check("polar_autotune", _lib.polar_autotune(
        fs.handle, int(nframes), _ptr(llr), _ptr(fval), _ptr(xhat), FKIND[fkind], PREC[prec],
        _stream(stream), C.byref(t), C.byref(fu), C.byref(ms)))
    return t.value, fu.value, ms.value


def polar_tune_save(path: str):
    _check("polar_tune_save", _lib.polar_tune_save(path.encode()))


def polar_tune_load(path: str) -> bool:
    rc = _lib.polar_tune_load(path.encode())
    if rc == POLAR_ENOTFOUND:
        return False
    _check("polar_tune_load", rc)
    return True


def polar_tune_clear():
    _lib.polar_tune_clear()


# ------------------------------------------------------------------ serving
class Server:
    """Owner of a library request server (destroyed on close / collection)."""

    def __init__(self, device=0, max_inflight=32, max_queue=4096, mem_budget=8 << 30,
                 fkind="minsum", prec="fp32", threads=0, persistent=False, max_log2n=0):
        cfg = ServerConfig(int(device), int(max_inflight), int(max_queue), int(mem_budget),
                           FKIND[fkind], PREC[prec], int(threads), int(bool(persistent)),
                           int(max_log2n))
        h = C.c_void_p()
        _check("polar_server_create", _lib.polar_server_create(C.byref(cfg), C.byref(h)))
        self.handle = h

    def submit(self, fs, nframes, llr, fval, xhat, uhat=None):
        """Ticket, or None when admission is refused (queue full)."""
        req = Request(fs.handle.value, int(nframes), llr.data_ptr(), fval.data_ptr(),
                      xhat.data_ptr(), uhat.data_ptr() if uhat is not None else None)
        t = C.c_uint64()
        rc = _lib.polar_server_submit(self.handle, C.byref(req), C.byref(t))
        if rc == POLAR_EBUSY:
            return None
        _check("polar_server_submit", rc)
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, queue_ms, latency_ms)."""
        r = Result()
        rc = _lib.polar_server_poll(self.handle, int(ticket), C.byref(r))
        if rc == POLAR_PENDING:
            return None
        if rc == POLAR_ENOTFOUND:
            raise PolarError("polar_server_poll", rc)
        return (r.status, r.queue_ms, r.latency_ms)

    def wait(self, ticket, timeout_ms=60000.0):
        r = Result()
        rc = _lib.polar_server_wait(self.handle, int(ticket), float(timeout_ms), C.byref(r))
        if rc == POLAR_ETIMEDOUT:
            raise PolarError("polar_server_wait", rc)
        if rc == POLAR_ENOTFOUND:
            raise PolarError("polar_server_wait", rc)
        return (r.status, r.queue_ms, r.latency_ms)

    def cancel(self, ticket):
        """True when the request was withdrawn before it ran (poll / wait then
        report POLAR_ECANCELED), False when it already runs or has finished."""
        rc = _lib.polar_server_cancel(self.handle, int(ticket))
        if rc == POLAR_EBUSY:
            return False
        _check("polar_server_cancel", rc)
        return True

    def stats(self):
        a, b, c, d = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_size_t()
        _check("polar_server_stats", _lib.polar_server_stats(self.handle, C.byref(a),
                                                             C.byref(b), C.byref(c), C.byref(d)))
        return {"launched": a.value, "completed": b.value, "refused": c.value,
                "scratch_bytes": d.value}

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.polar_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def polar_server_create(**kw) -> Server:
    return Server(**kw)


def polar_static_scratch_bytes() -> int:
    return int(_lib.polar_static_scratch_bytes())


def exported_symbols():
    """Names of the C ABI functions the binding declares."""
    return [n for n in dir(_lib) if n.startswith("polar_")]
