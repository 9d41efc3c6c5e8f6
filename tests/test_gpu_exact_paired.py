"""Paired exact-f comparison at the size of Table 1's first row.

Sec. 4 decodes with the phi-based update (exact f); Table 1's first row is
the BSC at p = 2 % with N = 2^16 and a frozen set whose information bits have
a summed error probability of at most 0.1 (Sec. 3).  The GPU's float32 exact
f and the float64 exact-f oracle decode the SAME seeded frames, and their
frame errors are compared pairwise: the discordant frames (one side wrong,
the other right) must be balanced within two standard errors (McNemar), and
the per-frame bit error rates must agree within two standard errors of their
paired differences.  Both sides build the degraded-channel frozen set on
their own and the masks are asserted equal first.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402

DEV = "cuda:0"
FRAMES = 256


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


def test_exact_f_paired_with_float64_oracle_table1_bsc_n16(P):
    n, p = 16, 0.02
    N = 1 << n
    w = S.Workload("table1_bsc_p02_n16", "bsc", p, n, 0.0, FRAMES, 0x7AB1E)
    fs = P.polar_build_frozen_set_tv(n, "bsc", p, 16, 0.0, 0.1)
    ofz, oK, osum = O.frozen_set_tv(n, "bsc", p, 0.0, 0.1, 16)
    assert fs.K == oK
    assert np.array_equal(S.unpack_bits(fs.mask(), N), ofz)
    assert osum <= 0.1

    x, y = S.frames(w, 0, FRAMES)
    xd = torch.from_numpy(x.view(np.int32)).to(DEV)
    fv = torch.empty_like(xd)
    P.polar_reveal(fs, FRAMES, xd, fv)
    llr = torch.empty(FRAMES, N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel("bsc", p, torch.from_numpy(y.view(np.int32)).to(DEV), llr)
    xh = torch.zeros_like(xd)
    P.polar_sc_decode_many(fs, FRAMES, llr, fv, xh, None, "exact", "fp32")
    torch.cuda.synchronize()
    xh = xh.cpu().numpy().view(np.uint32)

    e_g, e_o, ber_g, ber_o = [], [], [], []
    for f in range(FRAMES):
        xb = S.unpack_bits(x[f], N)
        gx = S.unpack_bits(xh[f], N)
        _, ox, _ = O.decode_frame("bsc", p, x[f], y[f], ofz, "exact", 64)
        e_g.append(int(not np.array_equal(gx, xb)))
        e_o.append(int(not np.array_equal(ox, xb)))
        ber_g.append(float(np.mean(gx != xb)))
        ber_o.append(float(np.mean(ox != xb)))
    e_g, e_o = np.array(e_g), np.array(e_o)
    fer_o = e_o.mean()
    # the code works as Table 1's row does: a frame error rate near the bound
    assert 0.01 <= fer_o <= 0.3, fer_o
    # McNemar: frames wrong on one side only are balanced
    b = int(((e_g == 1) & (e_o == 0)).sum())
    c = int(((e_g == 0) & (e_o == 1)).sum())
    assert abs(b - c) <= 2.0 * math.sqrt(max(b + c, 1)), (b, c)
    # paired per-frame bit error rates
    d = np.array(ber_g) - np.array(ber_o)
    se = float(np.std(d, ddof=1)) / math.sqrt(FRAMES) if np.any(d) else 0.0
    assert abs(float(d.mean())) <= 2.0 * se + 1e-12, (d.mean(), se)
