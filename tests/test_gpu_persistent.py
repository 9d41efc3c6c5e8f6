"""Persistent decoder (one launch, whole frames per CTA from a device queue)
through the C ABI.

Bar: float32 min-sum x_hat / u_hat bit-exact with the CPU oracle for frames
of mixed lengths and codes in one launch (ragged queues longer than the
grid, codes with rate-0 nodes above the subtree size, codes shorter than a
word); exact f bit-identical to the launched schedule, which performs the
same float32 operations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


@pytest.fixture(autouse=True)
def default_config(P):
    saved = {k: P.polar_config_get(k)
             for k in ("persist_log2", "persistent", "subtree_log2", "autotune")}
    yield
    for k, v in saved.items():
        P.polar_config_set(k, v)


def to_dev_words(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(DEV)


def words_np(t):
    return t.cpu().numpy().view(np.uint32)


def make_mask(rng, n, kind):
    N = 1 << n
    if kind == "random":
        return (rng.random(N) < 0.5).astype(np.uint8)
    if kind == "all_frozen":
        return np.ones(N, np.uint8)
    if kind == "all_info":
        return np.zeros(N, np.uint8)
    if kind == "front_frozen":      # first half frozen: a rate-0 child at the top
        fz = (rng.random(N) < 0.3).astype(np.uint8)
        fz[: N // 2] = 1
        return fz
    if kind == "low_rate":          # GA set far below capacity: many rate-0 nodes
        return O.frozen_set(n, "biawgn", 4.0, 0.05)[0]
    return O.frozen_set(n, "bsc", 0.05, 0.6)[0]


def make_frames(P, rng, specs, uhat_every=2):
    """specs: list of (n, kind, llr_kind).  Returns (frames, inputs)."""
    frames, inputs = [], []
    masks = {}
    for j, (n, kind, llr_kind) in enumerate(specs):
        N = 1 << n
        if (n, kind) not in masks:
            fz = make_mask(rng, n, kind)
            masks[(n, kind)] = (fz, P.polar_frozen_set_from_mask(n, S.pack_bits(fz)))
        fz, fs = masks[(n, kind)]
        if llr_kind == "gauss":
            L = rng.normal(0.5, 2.0, N).astype(np.float32)
        else:                       # +-c with many exact ties in g
            L = (np.float32(2.5) * (1 - 2 * (rng.random(N) < 0.1))).astype(np.float32)
        fvb = (rng.integers(0, 2, N) * fz).astype(np.uint8)
        llr = torch.from_numpy(L).to(DEV)
        fv = to_dev_words(S.pack_bits(fvb))
        xh = torch.full_like(fv, -1)
        uh = torch.full_like(fv, -1) if j % uhat_every == 0 else None
        frames.append((fs, llr, fv, xh, uh))
        inputs.append((L, fz, fvb))
    return frames, inputs


def check_against_oracle(frames, inputs, fkind="minsum"):
    for (fs, _, _, xh, uh), (L, fz, fvb) in zip(frames, inputs):
        ou, ox = O.sc_decode(L, fz, fvb, fkind)
        N = fs.N
        assert np.array_equal(S.unpack_bits(words_np(xh), N), ox), (fs.log2n,)
        if uh is not None:
            assert np.array_equal(S.unpack_bits(words_np(uh), N), ou), (fs.log2n,)


SPECS = [(n, kind, lk)
         for n in (1, 3, 5, 8, 12, 13, 14, 16)
         for kind in ("polar", "random", "all_info", "all_frozen", "front_frozen")
         for lk in ("gauss", "bsc")]


@pytest.mark.parametrize("t", [5, 9, 13])
def test_persistent_mixed_minsum_bitexact(P, t):
    P.polar_config_set("persist_log2", t)
    rng = np.random.default_rng(100 + t)
    frames, inputs = make_frames(P, rng, SPECS)
    P.polar_sc_decode_persistent(frames)
    torch.cuda.synchronize()
    check_against_oracle(frames, inputs)


@pytest.mark.parametrize("t", [6, 10])
def test_persistent_rate0_upper_nodes(P, t):
    """Low-rate and front-frozen codes: rate-0 nodes and skipped f / g steps
    above the subtree size."""
    P.polar_config_set("persist_log2", t)
    rng = np.random.default_rng(7 + t)
    specs = [(16, "low_rate", "gauss"), (15, "front_frozen", "bsc"), (16, "low_rate", "bsc"),
             (12, "front_frozen", "gauss")]
    frames, inputs = make_frames(P, rng, specs, uhat_every=1)
    P.polar_sc_decode_persistent(frames)
    torch.cuda.synchronize()
    check_against_oracle(frames, inputs)


def test_persistent_queue_longer_than_grid(P):
    """More frames than resident CTAs: CTAs loop over the queue.  Every frame
    equals the launched schedule's result; a sample equals the oracle."""
    P.polar_config_set("persist_log2", 9)
    rng = np.random.default_rng(11)
    specs = [(int(rng.choice([10, 11, 12])), "polar", "gauss") for _ in range(700)]
    frames, inputs = make_frames(P, rng, specs, uhat_every=3)
    P.polar_sc_decode_persistent(frames)
    torch.cuda.synchronize()
    for (fs, llr, fv, xh, uh) in frames:
        x2 = torch.full_like(xh, -1)
        u2 = torch.full_like(xh, -1) if uh is not None else None
        P.polar_sc_decode_many(fs, 1, llr, fv, x2, u2)
        torch.cuda.synchronize()
        assert torch.equal(x2, xh)
        if uh is not None:
            assert torch.equal(u2, uh)
    check_against_oracle(frames[:12], inputs[:12])


def test_persistent_exact_f_matches_launched(P):
    P.polar_config_set("persist_log2", 10)
    rng = np.random.default_rng(23)
    specs = [(n, "polar", "gauss") for n in (9, 12, 14, 15, 12, 10)]
    frames, _ = make_frames(P, rng, specs, uhat_every=1)
    P.polar_sc_decode_persistent(frames, fkind="exact")
    torch.cuda.synchronize()
    for (fs, llr, fv, xh, uh) in frames:
        x2, u2 = torch.full_like(xh, -1), torch.full_like(xh, -1)
        P.polar_sc_decode_many(fs, 1, llr, fv, x2, u2, "exact")
        torch.cuda.synchronize()
        assert torch.equal(x2, xh) and torch.equal(u2, uh)


def test_persistent_workload_2_20(P):
    """Eight frames of the 2^20 BSC workload next to four 2^16 frames."""
    P.polar_config_set("persist_log2", 13)
    w, w2 = S.WORKLOADS["bsc_p03_n20"], S.WORKLOADS["bsc_p02_n16"]
    frames, expect = [], []
    for wl, count in ((w, 8), (w2, 4)):
        fs = P.polar_build_frozen_set(wl.log2n, wl.channel, wl.param, wl.rate)
        ofz, _ = O.frozen_set(wl.log2n, wl.channel, wl.param, wl.rate)
        x, y = S.frames(wl, 0, count)
        xd = to_dev_words(x)
        fv = torch.empty_like(xd)
        P.polar_reveal(fs, count, xd, fv)
        llr = torch.empty(count, wl.N, dtype=torch.float32, device=DEV)
        P.polar_llr_from_channel("bsc", wl.param, to_dev_words(y), llr)
        xh = torch.full_like(xd, -1)
        for f in range(count):
            frames.append((fs, llr[f], fv[f], xh[f], None))
        expect.append((wl, fs, ofz, x, y, llr, fv, xh, count))
    P.polar_sc_decode_persistent(frames)
    torch.cuda.synchronize()
    for wl, fs, ofz, x, y, llr, fv, xh, count in expect:
        x2 = torch.full_like(xh, -1)
        P.polar_sc_decode_many(fs, count, llr, fv, x2, None)
        torch.cuda.synchronize()
        assert torch.equal(x2, xh)
        got = words_np(xh)
        for f in (0, count - 1):
            _, ox, _ = O.decode_frame(wl.channel, wl.param, x[f], y[f], ofz, "minsum", 32)
            assert np.array_equal(S.unpack_bits(got[f], wl.N), ox)


def test_decode_batch_takes_the_persistent_launch(P):
    rng = np.random.default_rng(31)
    specs = [(12, "polar", "gauss"), (14, "random", "bsc"), (10, "polar", "gauss")]
    frames, inputs = make_frames(P, rng, specs, uhat_every=2)
    P.polar_config_set("persistent", 1)
    before = P.polar_kernel_launches()
    P.polar_sc_decode_batch(frames)
    torch.cuda.synchronize()
    assert P.polar_kernel_launches() - before == 1
    check_against_oracle(frames, inputs)
    P.polar_config_set("persistent", 0)
    P.polar_config_set("subtree_log2", 9)           # several launches per frame
    for f in frames:
        f[3].fill_(-1)
    before = P.polar_kernel_launches()
    P.polar_sc_decode_batch(frames)
    torch.cuda.synchronize()
    assert P.polar_kernel_launches() - before > 3
    check_against_oracle(frames, inputs)


def test_upload_makes_a_code_resident_before_its_first_decode(P):
    """polar_frozen_set_upload is idempotent, refuses a device that does not
    exist, and a decode after it gives the oracle's bits."""
    P.polar_config_set("persist_log2", 9)
    rng = np.random.default_rng(77)
    frames, inputs = make_frames(P, rng, [(14, "polar", "gauss"), (12, "front_frozen", "bsc")],
                                 uhat_every=1)
    for fs, *_ in frames:
        P.polar_frozen_set_upload(fs)
        P.polar_frozen_set_upload(fs)
    with pytest.raises(P.PolarError):
        P.polar_frozen_set_upload(frames[0][0], torch.cuda.device_count())
    P.polar_sc_decode_persistent(frames)
    torch.cuda.synchronize()
    check_against_oracle(frames, inputs)


@pytest.mark.parametrize("prec", ["fp16", "int8"])
@pytest.mark.parametrize("fkind", ["minsum", "exact"])
@pytest.mark.parametrize("t", [9, 13])
def test_reduced_storage_persistent(P, prec, fkind, t):
    """FP16 / INT8 levels in the persistent decoder: bit-identical to the
    launched schedule at the same subtree size (the levels >= t stored and
    rounded alike, int8 with the same per-frame scale), and min-sum equal to
    the oracle's storage model."""
    rng = np.random.default_rng(500 + t)
    specs = [(n, kind, "gauss") for n in (5, 9, 12, 14, 16) for kind in ("polar", "random")]
    specs += [(15, "front_frozen", "bsc"), (13, "low_rate", "gauss")]
    frames, inputs = make_frames(P, rng, specs)
    P.polar_config_set("persist_log2", t)
    P.polar_sc_decode_persistent(frames, fkind=fkind, prec=prec)
    torch.cuda.synchronize()
    P.polar_config_set("autotune", 0)
    P.polar_config_set("subtree_log2", t)
    try:
        target = P.polar_config_get("int8_target")
        for (fs, llr, fv, xh, uh), (L, fz, fvb) in zip(frames, inputs):
            rx, ru = torch.full_like(fv, -1), torch.full_like(fv, -1)
            P.polar_sc_decode_many(fs, 1, llr, fv, rx, ru, fkind, prec)
            torch.cuda.synchronize()
            assert torch.equal(xh, rx), (fs.log2n, prec, fkind)
            if uh is not None:
                assert torch.equal(uh, ru), (fs.log2n, prec, fkind)
            if fkind == "minsum":
                sc = O.int8_scale(L, target) if prec == "int8" else 1.0
                ou, ox = O.sc_decode_store(L, fz, fvb, "minsum", prec, sc,
                                           min_level=min(fs.log2n, t))
                assert np.array_equal(S.unpack_bits(words_np(xh), fs.N), ox), fs.log2n
    finally:
        P.polar_config_set("autotune", 1)
