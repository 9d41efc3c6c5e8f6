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


def inputs(P, w, first, count):
    fs = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    x, y = S.frames(w, first, count)
    xd = torch.from_numpy(x.view(np.int32)).to(DEV)
    fv = torch.empty_like(xd)
    P.polar_reveal(fs, count, xd, fv)
    llr = torch.empty(count, w.N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel(w.channel, w.param, torch.from_numpy(y.view(np.int32)).to(DEV), llr)
    return fs, llr, fv


@pytest.mark.parametrize("fkind", ["minsum", "exact"])
def test_noalloc_matches_regular_decode_twice(P, fkind):
    w = S.WORKLOADS["bsc_p03_n20"]
    stream = torch.cuda.Stream()
    for call, first in enumerate((0, 3)):          # two calls in a row, new data each
        fs, llr, fv = inputs(P, w, first, 3)
        ref_x = torch.zeros_like(fv)
        ref_u = torch.zeros_like(fv)
        P.polar_sc_decode_many(fs, 3, llr, fv, ref_x, ref_u, fkind, "fp32", stream)
        got_x = torch.full_like(fv, -1)
        got_u = torch.full_like(fv, -1)
        P.polar_sc_decode_many_noalloc(fs, 3, llr, fv, got_x, got_u, fkind, "fp32", stream)
        stream.synchronize()
        assert torch.equal(got_x, ref_x), f"x_hat differs on call {call}"
        assert torch.equal(got_u, ref_u), f"u_hat differs on call {call}"


def test_noalloc_rejects_oversize_request(P):
    w = S.WORKLOADS["bsc_p03_n20"]
    fs = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    need = 64 * (w.N - (1 << 13)) * 4
    assert need > P.polar_static_scratch_bytes()
    llr = torch.empty(16, dtype=torch.float32, device=DEV)
    words = torch.empty(16, dtype=torch.int32, device=DEV)
    rc = P.lib().polar_sc_decode_many_noalloc(fs.handle, 64, llr.data_ptr(), words.data_ptr(),
                                              words.data_ptr(), None, 0, 0, None)
    assert rc == P.POLAR_EINVAL
    assert "static array" in P.lib().polar_last_error_string().decode()
