"""Seeded synthetic inputs for SC polar decoding in syndrome form.

This module only draws random numbers and lays them out.  It holds none of
the decoder's arithmetic: no transform, no LLR, no construction.  Both the
oracle-side tests and the CUDA path (tests and ``bench.py``) take their inputs
from here, so the two sides decode byte-identical inputs.

Generator: SplitMix64 (Steele, Lea & Flood, 2014) used as a counter-based
stream.  Stream (seed, frame, sid) has the key
``key = mix(seed * GAMMA + (frame << 8 | sid))`` and its i-th output
(i = 0, 1, ...) is ``mix(key + (i + 1) * GAMMA)`` with the SplitMix64
finaliser ``mix``; all arithmetic is modulo 2^64.

Draws (per frame f):
  * Alice's string x: stream sid=1, 64 uniform bits per output, packed
    little-endian into uint32 words (bit i = word i // 32, bit i % 32);
  * BSC errors e_i ~ Bernoulli(p): stream sid=2, ``(r >> 11) * 2^-53 < p``;
    Bob's y = x XOR e (packed bits);
  * BIAWGN noise: stream sid=3, Box-Muller (1958) on output pairs
    (r0, r1): u1 = ((r0 >> 11) + 1) 2^-53, u2 = (r1 >> 11) 2^-53,
    z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2);
    Bob's y_i = (1 - 2 x_i) + sigma z_i in float64.

The workloads are the ones the paper measures (Table 1: BSC at 2 % QBER and
the BI-AWGN channel near SNR 1, block sizes 2^16 .. 2^24), which are
themselves synthetic in the paper; no dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_U64 = np.uint64


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(_M1)
        z = (z ^ (z >> _U64(27))) * _U64(_M2)
        return z ^ (z >> _U64(31))


def stream(seed: int, frame: int, sid: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 stream (seed, frame, sid)."""
    k0 = (seed * GAMMA + ((frame << 8) | sid)) & 0xFFFFFFFFFFFFFFFF
    key = _mix(np.array([k0], dtype=np.uint64))[0]
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = key + idx * _U64(GAMMA)
    return _mix(ctr)


def uniform53(r: np.ndarray) -> np.ndarray:
    return (r >> _U64(11)).astype(np.float64) * (2.0 ** -53)


def alice_bits(seed: int, frame: int, N: int) -> np.ndarray:
    """Alice's uniform string x, packed: uint32[N/32] (N >= 32)."""
    if N < 64:
        r = stream(seed, frame, 1, 1)
        w = r.view(np.uint32)[: max(1, N // 32)].copy()
        if N < 32:
            w &= np.uint32((1 << N) - 1)
        return w
    return stream(seed, frame, 1, N // 64).view(np.uint32).copy()


def bsc_errors(seed: int, frame: int, N: int, p: float) -> np.ndarray:
    """Error pattern e_i ~ Bernoulli(p), packed uint32[ceil(N/32)]."""
    e = uniform53(stream(seed, frame, 2, N)) < p
    return pack_bits(e)


def gaussian(seed: int, frame: int, N: int) -> np.ndarray:
    """N standard normal draws (Box-Muller on consecutive output pairs)."""
    M = (N + 1) // 2
    r = stream(seed, frame, 3, 2 * M)
    u1 = ((r[0::2] >> _U64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (r[1::2] >> _U64(11)).astype(np.float64) * (2.0 ** -53)
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * M, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:N]


def pack_bits(b: np.ndarray) -> np.ndarray:
    """Bool/0-1 array -> little-endian packed uint32 words."""
    b = np.asarray(b, dtype=np.uint8).reshape(-1)
    nw = (b.size + 31) // 32
    pad = np.zeros(nw * 32, dtype=np.uint8)
    pad[: b.size] = b
    return np.packbits(pad, bitorder="little").view(np.uint32).copy()


def unpack_bits(w: np.ndarray, N: int) -> np.ndarray:
    """Packed uint32 words -> uint8 0/1 array of length N."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.uint32).reshape(-1))
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:N].copy()


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: a channel, a code and a number of frames."""
    name: str
    channel: str          # "bsc" or "biawgn"
    param: float          # p for the BSC, sigma^2 for the BI-AWGN channel
    log2n: int
    rate: float           # K = floor(rate * N)
    frames: int
    seed: int

    @property
    def N(self) -> int:
        return 1 << self.log2n

    @property
    def K(self) -> int:
        return int(math.floor(self.rate * self.N))


# Workloads shaped like the paper's Table 1 rows (BSC 2-3 % and BI-AWGN near
# SNR 1, N = 2^16 .. 2^24), with the rates fixed per workload.
WORKLOADS = {
    "bsc_p02_n16": Workload("bsc_p02_n16", "bsc", 0.02, 16, 0.80, 100, 0x5EED + 1),
    "bsc_p03_n20": Workload("bsc_p03_n20", "bsc", 0.03, 20, 0.75, 64, 0x5EED + 2),
    "biawgn_s1_n24": Workload("biawgn_s1_n24", "biawgn", 1.0, 24, 0.44, 16, 0x5EED + 3),
    "prec_biawgn_n22": Workload("prec_biawgn_n22", "biawgn", 1.0, 22, 0.44, 1000, 0x5EED + 5),
    "prec_bsc_n22": Workload("prec_bsc_n22", "bsc", 0.02, 22, 0.82, 1000, 0x5EED + 6),
}


def frame(w: Workload, f: int):
    """Inputs of frame f: (x packed uint32[N/32], y).

    y is packed uint32[N/32] for the BSC and float64[N] for the BI-AWGN.
    """
    N = w.N
    x = alice_bits(w.seed, f, N)
    if w.channel == "bsc":
        return x, x ^ bsc_errors(w.seed, f, N, w.param)
    xb = unpack_bits(x, N).astype(np.float64)
    y = (1.0 - 2.0 * xb) + math.sqrt(w.param) * gaussian(w.seed, f, N)
    return x, y


def frames(w: Workload, first: int, count: int):
    """Stacked inputs of frames first .. first+count-1: (x [F, N/32], y [F, ...])."""
    xs, ys = [], []
    for f in range(first, first + count):
        x, y = frame(w, f)
        xs.append(x)
        ys.append(y)
    return np.stack(xs), np.stack(ys)


# ------------------------------------------------------------------ device-side draws
# For streams too large to draw on the host (the served mixed workload), the
# same distributions are drawn on the GPU with torch's Philox generator,
# seeded per request.  Only random draws and bit packing happen here.
def _gen(seed: int, idx: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(_mix(np.array([(seed * GAMMA + idx) & 0xFFFFFFFFFFFFFFFF],
                                    dtype=np.uint64))[0]) & 0x7FFFFFFFFFFFFFFF)
    return g


def pack_bits_torch(bits):
    """bool/0-1 tensor [..., N] -> int32 words [..., N/32] (little-endian)."""
    import torch
    b = bits.to(torch.int64).reshape(*bits.shape[:-1], -1, 32)
    w = (b << torch.arange(32, device=bits.device, dtype=torch.int64)).sum(-1)
    return (w & 0xFFFFFFFF).to(torch.int64).where(w < 2 ** 31, w - 2 ** 32).to(torch.int32)


def unpack_bits_torch(words, N: int):
    import torch
    w = words.to(torch.int64) & 0xFFFFFFFF
    b = (w.unsqueeze(-1) >> torch.arange(32, device=words.device, dtype=torch.int64)) & 1
    return b.reshape(*words.shape[:-1], -1)[..., :N]


def device_frame(channel: str, param: float, N: int, seed: int, idx: int, device):
    """(x words int32 [N/32], y) on the device: y packed int32 words (BSC) or
    float64 [N] (BI-AWGN, y = (1 - 2x) + sqrt(sigma^2) z)."""
    import torch
    g = _gen(seed, idx, device)
    xb = torch.randint(0, 2, (N,), generator=g, device=device, dtype=torch.int32)
    x = pack_bits_torch(xb)
    if channel == "bsc":
        e = torch.rand(N, generator=g, device=device, dtype=torch.float64) < param
        return x, pack_bits_torch(xb.bool() ^ e)
    z = torch.randn(N, generator=g, device=device, dtype=torch.float64)
    return x, (1.0 - 2.0 * xb.to(torch.float64)) + math.sqrt(param) * z
