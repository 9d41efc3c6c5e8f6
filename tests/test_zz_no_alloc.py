"""The allocation-free decode entry point against the regular one.

polar_sc_decode_many_noalloc serves callers that cannot allocate device
memory (a framework pool owns it all, or cudaMalloc's implicit
synchronisation is not acceptable in their loop).  It keeps its scratch in a
fixed device array inside the library.  This file is collected last so that a
run stopping at the first failure has run every other test before it; it
passes alone in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1204_5882_gb300 import synth as S  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    saved = {k: polar.polar_config_get(k) for k in ("subtree_log2", "shortcuts")}
    polar.polar_config_set("subtree_log2", 13)
    polar.polar_config_set("shortcuts", 1)
    yield polar
    for k, v in saved.items():
        polar.polar_config_set(k, v)


_codes = {}


def code(P, w):
    key = (w.log2n, w.channel, w.param, w.rate)
    if key not in _codes:
        _codes[key] = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    return _codes[key]


def inputs(P, w, first, count):
    fs = code(P, w)
    x, y = S.frames(w, first, count)
    xd = torch.from_numpy(x.view(np.int32)).to(DEV)
    fv = torch.empty_like(xd)
    P.polar_reveal(fs, count, xd, fv)
    llr = torch.empty(count, w.N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel(w.channel, w.param, torch.from_numpy(y.view(np.int32)).to(DEV), llr)
    return fs, llr, fv


def both(P, fs, count, llr, fv, fkind, prec, stream):
    """(regular x, u), (allocation-free x, u) on the same inputs."""
    ref_x = torch.zeros_like(fv)
    ref_u = torch.zeros_like(fv)
    P.polar_sc_decode_many(fs, count, llr, fv, ref_x, ref_u, fkind, prec, stream)
    got_x = torch.full_like(fv, -1)
    got_u = torch.full_like(fv, -1)
    P.polar_sc_decode_many_noalloc(fs, count, llr, fv, got_x, got_u, fkind, prec, stream)
    stream.synchronize()
    return (ref_x, ref_u), (got_x, got_u)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "int8"])
@pytest.mark.parametrize("fkind", ["minsum", "exact"])
def test_noalloc_matches_regular_decode_twice(P, fkind, prec):
    w = S.WORKLOADS["bsc_p03_n20"]
    stream = torch.cuda.Stream()
    for call, first in enumerate((0, 3)):          # two calls in a row, new data each
        fs, llr, fv = inputs(P, w, first, 3)
        (rx, ru), (gx, gu) = both(P, fs, 3, llr, fv, fkind, prec, stream)
        assert torch.equal(gx, rx), f"x_hat differs on call {call}"
        assert torch.equal(gu, ru), f"u_hat differs on call {call}"


@pytest.mark.parametrize("shortcuts", [1, 0])
def test_noalloc_consecutive_calls_on_different_codes(P, shortcuts):
    """A call on one code leaves its mask, class table and levels in the
    array; the next call, on another code and length, must not see them."""
    small = S.Workload("n16", "bsc", 0.02, 16, 0.80, 4, 0x5EED + 71)
    large = S.WORKLOADS["bsc_p03_n20"]
    P.polar_config_set("shortcuts", shortcuts)
    try:
        stream = torch.cuda.Stream()
        for step, (w, count, prec) in enumerate(((small, 4, "fp32"), (large, 2, "fp32"),
                                                 (small, 4, "int8"), (large, 3, "fp16"),
                                                 (small, 2, "fp32"))):
            fs, llr, fv = inputs(P, w, step, count)
            (rx, ru), (gx, gu) = both(P, fs, count, llr, fv, "minsum", prec, stream)
            assert torch.equal(gx, rx), f"x_hat differs at step {step}"
            assert torch.equal(gu, ru), f"u_hat differs at step {step}"
    finally:
        P.polar_config_set("shortcuts", 1)


def test_noalloc_largest_documented_requests(P):
    """The header's largest examples fit and decode equal to the regular
    path; one frame more is refused before any launch."""
    stream = torch.cuda.Stream()
    w21 = S.Workload("n21", "bsc", 0.03, 21, 0.75, 2, 0x5EED + 72)
    fs, llr, fv = inputs(P, w21, 0, 2)
    (rx, ru), (gx, gu) = both(P, fs, 1, llr[:1], fv[:1], "minsum", "fp32", stream)
    assert torch.equal(gx, rx) and torch.equal(gu, ru)
    out2 = torch.zeros_like(fv)                      # sized for both frames
    rc = P.lib().polar_sc_decode_many_noalloc(fs.handle, 2, llr.data_ptr(), fv.data_ptr(),
                                              out2.data_ptr(), None, 0, 0, None)
    assert rc == P.POLAR_EINVAL
    w20 = S.WORKLOADS["bsc_p03_n20"]
    fs, llr, fv = inputs(P, w20, 0, 16)
    (rx, ru), (gx, gu) = both(P, fs, 15, llr[:15], fv[:15], "minsum", "int8", stream)
    assert torch.equal(gx, rx) and torch.equal(gu, ru)
    out16 = torch.zeros_like(fv)                     # sized for all 16 frames
    rc = P.lib().polar_sc_decode_many_noalloc(fs.handle, 16, llr.data_ptr(), fv.data_ptr(),
                                              out16.data_ptr(), None, 0, 2, None)
    assert rc == P.POLAR_EINVAL


def test_noalloc_leaves_free_device_memory_unchanged(P):
    w = S.WORKLOADS["bsc_p03_n20"]
    stream = torch.cuda.Stream()
    fs, llr, fv = inputs(P, w, 0, 3)
    xh = torch.zeros_like(fv)
    uh = torch.zeros_like(fv)
    P.polar_sc_decode_many_noalloc(fs, 3, llr, fv, xh, uh, "minsum", "fp32", stream)
    stream.synchronize()                             # first call: address lookup done
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        P.polar_sc_decode_many_noalloc(fs, 3, llr, fv, xh, uh, "exact", "fp32", stream)
    stream.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversize_request(P):
    w = S.WORKLOADS["bsc_p03_n20"]
    fs = code(P, w)
    need = 64 * (w.N - (1 << 13)) * 4
    assert need > P.polar_static_scratch_bytes()
    # buffers sized for all 64 frames, although the call is refused first
    llr = torch.zeros(64, w.N, dtype=torch.float32, device=DEV)
    fv = torch.zeros(64, w.N // 32, dtype=torch.int32, device=DEV)
    xh = torch.zeros_like(fv)
    rc = P.lib().polar_sc_decode_many_noalloc(fs.handle, 64, llr.data_ptr(), fv.data_ptr(),
                                              xh.data_ptr(), None, 0, 0, None)
    assert rc == P.POLAR_EINVAL
    assert "static array" in P.lib().polar_last_error_string().decode()
