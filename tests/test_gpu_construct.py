"""Frozen-set construction on the GPU in double precision against the oracle.

Sec. 3 freezes the least reliable bit-channels; the device builds the same
reliabilities as the oracle (Bhattacharyya for the BSC, the Gaussian
approximation for the BI-AWGN channel) and ranks them with the same tie rule
(the lower index frozen first).  Its exp / log / pow round differently from
the host's, so the masks must agree everywhere except at bit-channels whose
reliability is within rounding of the cut; with Sec. 3's sum rule K may move
by one only where the summed error probability meets the budget within
rounding.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402

REL = 1e-9            # relative closeness that counts as "within rounding"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


def near(a, b):
    return abs(a - b) <= REL * max(1.0, abs(a), abs(b))


def check_masks(lb, fz_o, fz_d, K):
    """Positions where the masks differ lie at the cut: their reliability is
    within rounding of the last information bit or the first frozen bit of
    the oracle's ranking (ascending ln P_e, higher index first on ties)."""
    N = lb.size
    order = np.lexsort((-np.arange(N), lb))      # ascending lb, then descending index
    edge = [lb[order[K - 1]]] if K > 0 else []
    if K < N:
        edge.append(lb[order[K]])
    diff = np.nonzero(fz_o != fz_d)[0]
    for i in diff:
        assert any(near(lb[i], e) for e in edge), (int(i), float(lb[i]), edge)
    return diff.size


CASES = [("bsc", 0.02, 10), ("bsc", 0.03, 16), ("bsc", 0.05, 20),
         ("biawgn", 1.0, 12), ("biawgn", 1.0 / 1.097, 18), ("biawgn", 4.0, 20)]


@pytest.mark.parametrize("ch,param,n", CASES)
def test_device_construction_rate_rule(P, ch, param, n):
    N = 1 << n
    lb = O.unreliability(n, ch, param)
    for R in (0.3, 0.5, 0.8):
        K = int(math.floor(R * N))
        fz_o = O.select_frozen(lb, K)
        fs = P.polar_build_frozen_set_device(n, ch, param, R, 0.0)
        assert fs.K == K
        fz_d = S.unpack_bits(fs.mask(), N)
        assert int((fz_d == 0).sum()) == K
        assert check_masks(lb, fz_o, fz_d, K) <= 4


@pytest.mark.parametrize("ch,param,n", CASES)
def test_device_construction_sum_rule(P, ch, param, n):
    N = 1 << n
    lb = O.unreliability(n, ch, param)
    fz_o, K_o, s_o = O.frozen_set_sum(n, ch, param, 0.1)
    fs = P.polar_build_frozen_set_device(n, ch, param, 0.0, 0.1)
    fz_d = S.unpack_bits(fs.mask(), N)
    assert int((fz_d == 0).sum()) == fs.K
    if fs.K != K_o:
        # only where the running sum meets the budget within rounding
        assert abs(fs.K - K_o) == 1
        pe = np.sort(np.exp(lb))
        acc = np.cumsum(pe)
        assert near(acc[min(fs.K, K_o)], 0.1) or near(acc[min(fs.K, K_o) - 1], 0.1)
    assert fs.sum_pe <= 0.1 * (1 + REL)
    if K_o > 0 and fs.K == K_o:
        assert fs.sum_pe == pytest.approx(s_o, rel=1e-6)
    assert check_masks(lb, fz_o, fz_d, min(fs.K, K_o)) <= 4


def test_device_construction_decodes_like_the_host_set(P):
    """A device-built set is a working frozen set: the 2^16 workload decodes
    bit-exact against the oracle with it (masks compared first)."""
    w = S.WORKLOADS["bsc_p02_n16"]
    fs_h = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    fs_d = P.polar_build_frozen_set_device(w.log2n, w.channel, w.param, w.rate, 0.0)
    assert np.array_equal(fs_h.mask(), fs_d.mask())
    x, y = S.frames(w, 0, 8)
    xd = torch.from_numpy(x.view(np.int32)).to("cuda:0")
    fv = torch.empty_like(xd)
    P.polar_reveal(fs_d, 8, xd, fv)
    llr = torch.empty(8, w.N, dtype=torch.float32, device="cuda:0")
    P.polar_llr_from_channel("bsc", w.param, torch.from_numpy(y.view(np.int32)).to("cuda:0"),
                             llr)
    xh = torch.zeros_like(xd)
    P.polar_sc_decode_many(fs_d, 8, llr, fv, xh, None, "minsum", "fp32")
    torch.cuda.synchronize()
    xh = xh.cpu().numpy().view(np.uint32)
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    for f in range(8):
        _, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "minsum", 32)
        assert np.array_equal(S.unpack_bits(xh[f], w.N), ox)


def test_device_construction_rejects_bad_arguments(P):
    for args in ((0, "bsc", 0.1, 0.5, 0.0), (28, "bsc", 0.1, 0.5, 0.0),
                 (10, "bsc", 0.6, 0.5, 0.0), (10, "biawgn", -1.0, 0.5, 0.0),
                 (10, "bsc", 0.1, 1.5, 0.0), (10, "bsc", 0.1, 0.0, -1.0)):
        with pytest.raises(P.PolarError) as e:
            P.polar_build_frozen_set_device(*args)
        assert e.value.status == P.POLAR_EINVAL
