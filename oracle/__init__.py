"""Python view of the plain C oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product path.  It shares
no code with the CUDA library; the only inputs both sides see come from
``paper_1204_5882_gb300.synth`` (random draws, no method arithmetic).

Every function below marshals numpy arrays (one bit per uint8) into the C
routines, whose comments cite the passage of the paper they follow.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.or_encode.argtypes = [P, C.c_int]
        for nm in ("or_llr_bsc_f32", "or_llr_bsc_f64", "or_llr_biawgn_f32", "or_llr_biawgn_f64"):
            getattr(L, nm).argtypes = [P, C.c_size_t, C.c_double, P]
        for nm, t in (("or_f_exact_f64", C.c_double), ("or_f_minsum_f64", C.c_double),
                      ("or_f_exact_f32", C.c_float), ("or_f_minsum_f32", C.c_float)):
            getattr(L, nm).argtypes = [t, t]
            getattr(L, nm).restype = t
        for nm in ("or_sc_decode_f64", "or_sc_decode_f32"):
            getattr(L, nm).argtypes = [C.c_int, C.c_int, P, P, P, P, P, P]
            getattr(L, nm).restype = C.c_int
        L.or_sc_decode_store.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, C.c_int, P, P, P,
                                         P, P, P]
        L.or_sc_decode_store.restype = C.c_int
        L.or_int8_scale.argtypes = [P, C.c_size_t, C.c_double]
        L.or_int8_scale.restype = C.c_float
        L.or_bhatt_log_from.argtypes = [C.c_int, C.c_double, P]
        L.or_bhatt_log_bsc.argtypes = [C.c_int, C.c_double, P]
        L.or_ga_lnphi.argtypes = [C.c_double]
        L.or_ga_lnphi.restype = C.c_double
        L.or_ga_lnphi_inv.argtypes = [C.c_double]
        L.or_ga_lnphi_inv.restype = C.c_double
        L.or_ga_mean.argtypes = [C.c_int, C.c_double, P]
        L.or_ga_lnpe.argtypes = [C.c_int, C.c_double, P]
        L.or_ln_q.argtypes = [C.c_double]
        L.or_ln_q.restype = C.c_double
        L.or_select_frozen.argtypes = [C.c_int, P, C.c_uint64, P]
        L.or_tv_pe.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, P]
        L.or_tv_pe.restype = C.c_int
        L.or_k_for_sum.argtypes = [C.c_int, P, C.c_double]
        L.or_k_for_sum.restype = C.c_uint64
        L.or_k_for_sum_log.argtypes = [C.c_int, P, C.c_double]
        L.or_k_for_sum_log.restype = C.c_uint64
        L.or_capacity_bsc.argtypes = [C.c_double]
        L.or_capacity_bsc.restype = C.c_double
        L.or_capacity_biawgn.argtypes = [C.c_double]
        L.or_capacity_biawgn.restype = C.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _bits(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def log2_of(N: int) -> int:
    n = int(N).bit_length() - 1
    if (1 << n) != N:
        raise ValueError("length must be a power of two")
    return n


# ---------------------------------------------------------------- transform
def encode(u) -> np.ndarray:
    """x = u F^{(x)n} (Sec. 3, natural order); F is an involution over GF(2)."""
    v = _bits(u).copy()
    lib().or_encode(_p(v), log2_of(v.size))
    return v


# ---------------------------------------------------------------- channel LLRs
def llr_bsc(y_bits, p: float, prec: int = 32) -> np.ndarray:
    y = _bits(y_bits)
    out = np.empty(y.size, dtype=np.float32 if prec == 32 else np.float64)
    getattr(lib(), f"or_llr_bsc_f{prec}")(_p(y), y.size, float(p), _p(out))
    return out


def llr_biawgn(y, sigma2: float, prec: int = 32) -> np.ndarray:
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    out = np.empty(y.size, dtype=np.float32 if prec == 32 else np.float64)
    getattr(lib(), f"or_llr_biawgn_f{prec}")(_p(y), y.size, float(sigma2), _p(out))
    return out


# ---------------------------------------------------------------- f and decoder
def f_exact(a: float, b: float, prec: int = 64) -> float:
    return getattr(lib(), f"or_f_exact_f{prec}")(a, b)


def f_minsum(a: float, b: float, prec: int = 64) -> float:
    return getattr(lib(), f"or_f_minsum_f{prec}")(a, b)


FKIND = {"minsum": 0, "exact": 1}


def sc_decode(llr, frozen, fval, fkind: str = "minsum", leaf: bool = False):
    """Recursive SC in syndrome form (Sec. 1, Sec. 4).

    ``llr`` float32 or float64 (selects the arithmetic), ``frozen``/``fval``
    one bit per uint8.  Returns (u_hat, x_hat) or (u_hat, x_hat, leaf_llr).
    """
    llr = np.ascontiguousarray(llr)
    prec = 32 if llr.dtype == np.float32 else 64
    if llr.dtype not in (np.float32, np.float64):
        raise TypeError("llr must be float32 or float64")
    n = log2_of(llr.size)
    fz, fv = _bits(frozen), _bits(fval)
    assert fz.size == llr.size and fv.size == llr.size
    u = np.empty(llr.size, dtype=np.uint8)
    x = np.empty(llr.size, dtype=np.uint8)
    lf = np.empty(llr.size, dtype=llr.dtype) if leaf else None
    rc = getattr(lib(), f"or_sc_decode_f{prec}")(
        n, FKIND[fkind], _p(llr), _p(fz), _p(fv), _p(u), _p(x),
        _p(lf) if leaf else None)
    if rc != 0:
        raise MemoryError("oracle decode failed")
    return (u, x, lf) if leaf else (u, x)


STORE = {"fp32": 0, "fp16": 1, "int8": 2}
INT8_TARGET = 8.0


def int8_scale(llr, target: float = INT8_TARGET) -> float:
    """Per-frame power-of-two scale so that mean |L| * scale is near target."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    return float(lib().or_int8_scale(_p(llr), llr.size, float(target)))


def sc_decode_store(llr, frozen, fval, fkind: str = "minsum", store: str = "fp16",
                    scale: float = 1.0, leaf: bool = False, min_level: int = 0):
    """SC with reduced-precision storage of the channel LLRs and of every
    level k >= min_level (float arithmetic; lower levels stay float)."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    n = log2_of(llr.size)
    fz, fv = _bits(frozen), _bits(fval)
    u = np.empty(llr.size, dtype=np.uint8)
    x = np.empty(llr.size, dtype=np.uint8)
    lf = np.empty(llr.size, dtype=np.float32) if leaf else None
    rc = lib().or_sc_decode_store(n, FKIND[fkind], STORE[store], float(scale), int(min_level),
                                  _p(llr), _p(fz), _p(fv), _p(u), _p(x),
                                  _p(lf) if leaf else None)
    if rc != 0:
        raise MemoryError("oracle decode failed")
    return (u, x, lf) if leaf else (u, x)


# ---------------------------------------------------------------- construction
def bhatt_log_from(n: int, lz0: float) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.float64)
    lib().or_bhatt_log_from(n, float(lz0), _p(out))
    return out


def bhatt_log_bsc(n: int, p: float) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.float64)
    lib().or_bhatt_log_bsc(n, float(p), _p(out))
    return out


def ga_lnphi(x: float) -> float:
    return lib().or_ga_lnphi(float(x))


def ga_lnphi_inv(t: float) -> float:
    return lib().or_ga_lnphi_inv(float(t))


def ga_mean(n: int, sigma2: float) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.float64)
    lib().or_ga_mean(n, float(sigma2), _p(out))
    return out


def ga_lnpe(n: int, sigma2: float) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.float64)
    lib().or_ga_lnpe(n, float(sigma2), _p(out))
    return out


def ln_q(x: float) -> float:
    return lib().or_ln_q(float(x))


def select_frozen(bad, K: int) -> np.ndarray:
    bad = np.ascontiguousarray(np.asarray(bad, dtype=np.float64))
    fz = np.empty(bad.size, dtype=np.uint8)
    lib().or_select_frozen(log2_of(bad.size), _p(bad), int(K), _p(fz))
    return fz


def tv_pe(n: int, channel: str, param: float, mu: int = 16) -> np.ndarray:
    """Upper bounds on every bit-channel's ML error probability from the
    degraded (Tal-Vardy) construction with mu output symbols per channel."""
    out = np.empty(1 << n, dtype=np.float64)
    rc = lib().or_tv_pe(n, 0 if channel == "bsc" else 1, float(param), int(mu), _p(out))
    if rc:
        raise ValueError((n, channel, param, mu))
    return out


def k_for_sum(bad, target: float) -> int:
    """Largest K whose K most reliable entries of `bad` sum to <= target."""
    bad = np.ascontiguousarray(np.asarray(bad, dtype=np.float64))
    return int(lib().or_k_for_sum(log2_of(bad.size), _p(bad), float(target)))


def k_for_sum_log(lbad, target: float) -> int:
    """k_for_sum on log-domain reliabilities (order by the logs, sum exp)."""
    lbad = np.ascontiguousarray(np.asarray(lbad, dtype=np.float64))
    return int(lib().or_k_for_sum_log(log2_of(lbad.size), _p(lbad), float(target)))


def frozen_set_sum(n: int, channel: str, param: float, sum_pe_max: float = 0.1):
    """(frozen mask, K, sum) of the Bhattacharyya (BSC) / GA (BI-AWGN) set
    whose K is chosen by Sec. 3's rule on those reliabilities."""
    lb = unreliability(n, channel, param)
    K = k_for_sum_log(lb, sum_pe_max)
    fz = select_frozen(lb, K)
    return fz, K, float(np.exp(lb[fz == 0]).sum())


def frozen_set_tv(n: int, channel: str, param: float, rate: float = 0.0,
                  sum_pe_max: float = 0.1, mu: int = 16):
    """(frozen mask, K, sum of P_e over the information set) of the degraded
    construction; K = floor(rate * N) if rate > 0, else the Sec. 3 rule."""
    pe = tv_pe(n, channel, param, mu)
    K = int(math.floor(rate * (1 << n))) if rate > 0 else k_for_sum(pe, sum_pe_max)
    fz = select_frozen(pe, K)
    return fz, K, float(pe[fz == 0].sum())


def unreliability(n: int, channel: str, param: float) -> np.ndarray:
    """ln Z (BSC, Bhattacharyya) or ln P_e (BI-AWGN, Gaussian approximation)."""
    if channel == "bsc":
        return bhatt_log_bsc(n, param)
    if channel == "biawgn":
        return ga_lnpe(n, param)
    raise ValueError(channel)


def frozen_set(n: int, channel: str, param: float, rate: float):
    """(frozen mask uint8[N], K) with K = floor(rate * N)."""
    N = 1 << n
    K = int(math.floor(rate * N))
    return select_frozen(unreliability(n, channel, param), K), K


def fer_bound(n: int, channel: str, param: float, frozen) -> float:
    """Sum over information bits of Z_i (BSC) or P_e,i (GA estimate), Sec. 3."""
    lb = unreliability(n, channel, param)
    info = np.asarray(frozen) == 0
    return float(np.exp(lb[info]).sum())


# ---------------------------------------------------------------- capacity
def capacity(channel: str, param: float) -> float:
    if channel == "bsc":
        return lib().or_capacity_bsc(float(param))
    return lib().or_capacity_biawgn(float(param))


def efficiency(K: int, N: int, channel: str, param: float) -> float:
    """beta = R / C (Sec. 2.1, Eq. 3 with I(x:y) = C for uniform x)."""
    return (K / N) / capacity(channel, param)


# ---------------------------------------------------------------- helpers
def unpack(w, N: int) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(w, dtype=np.uint32).reshape(-1))
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:N].copy()


def reveal(x_bits, frozen) -> np.ndarray:
    """Alice's side of syndrome reconciliation (Sec. 1): u = x F^{(x)n}
    (F is an involution), revealed at frozen positions, zero elsewhere."""
    u = encode(x_bits)
    return (u & _bits(frozen)).astype(np.uint8)


def decode_frame(channel: str, param: float, x_packed, y, frozen, fkind="minsum",
                 prec: int = 32):
    """Full oracle pipeline for one synthetic frame.

    Returns (u_hat, x_hat, x) as 0/1 uint8 arrays.
    """
    N = np.asarray(frozen).size
    x = unpack(x_packed, N)
    fv = reveal(x, frozen)
    if channel == "bsc":
        L = llr_bsc(unpack(y, N), param, prec)
    else:
        L = llr_biawgn(y, param, prec)
    u_hat, x_hat = sc_decode(L, frozen, fv, fkind)
    return u_hat, x_hat, x
