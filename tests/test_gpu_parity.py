"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bar: bit-exact x_hat and u_hat for float32 min-sum SC (every frame compared
element by element); bit-exact LLR maps, transforms and reveals; exact-f
frame error rate within two binomial standard errors of the float64 oracle.
Inputs come from the seeded generators in paper_1204_5882_gb300.synth; each
side builds its own frozen set and they are asserted equal first.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


DEV = "cuda:0"


def to_dev_words(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(DEV)


def words_np(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.fixture(autouse=True)
def default_config(P):
    saved = {k: P.polar_config_get(k)
             for k in ("subtree_log2", "shortcuts", "graphs", "plain", "fuse", "pdl",
                       "prologue", "split_log2", "autotune")}
    yield
    for k, v in saved.items():
        P.polar_config_set(k, v)


def gpu_decode(P, fs, llr_np, fv_words, fkind="minsum", prec="fp32", uhat=True):
    F = llr_np.shape[0]
    llr = torch.from_numpy(np.ascontiguousarray(llr_np, dtype=np.float32)).to(DEV)
    fv = to_dev_words(fv_words)
    xh = torch.full_like(fv, -1)
    uh = torch.full_like(fv, -1) if uhat else None
    P.polar_sc_decode_many(fs, F, llr, fv, xh, uh, fkind, prec)
    torch.cuda.synchronize()
    return words_np(xh), (words_np(uh) if uhat else None)


# ------------------------------------------------------------------ maps
def test_llr_bsc_bitexact(P):
    w = S.WORKLOADS["bsc_p02_n16"]
    x, y = S.frames(w, 0, 3)
    llr = torch.empty(3, w.N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel("bsc", w.param, to_dev_words(y), llr)
    got = llr.cpu().numpy()
    for f in range(3):
        assert np.array_equal(got[f], O.llr_bsc(S.unpack_bits(y[f], w.N), w.param, 32))


@pytest.mark.parametrize("count", [2 ** 16, 2 ** 16 + 1, 7])
def test_llr_biawgn_bitexact(P, count):
    rng = np.random.default_rng(3)
    y = rng.normal(1.0, 1.0, count)
    yd = torch.from_numpy(y).to(DEV)
    llr = torch.empty(count, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel("biawgn", 0.7, yd, llr)
    assert np.array_equal(llr.cpu().numpy(), O.llr_biawgn(y, 0.7, 32))


@pytest.mark.parametrize("n", [1, 3, 5, 6, 10, 17, 18, 22])
def test_encode_matches_oracle(P, n):
    N = 1 << n
    F = 3
    rng = np.random.default_rng(n)
    u = rng.integers(0, 2, (F, N)).astype(np.uint8)
    words = np.stack([S.pack_bits(r) for r in u])
    ud = to_dev_words(words)
    out = torch.zeros_like(ud)
    P.polar_encode(n, F, ud, out)
    got = words_np(out)
    for f in range(F):
        assert np.array_equal(S.unpack_bits(got[f], N), O.encode(u[f]))
    P.polar_encode(n, F, ud, ud)           # in place
    assert np.array_equal(words_np(ud), got)


def test_reveal_matches_oracle(P):
    n, F = 16, 4
    fs = P.polar_build_frozen_set(n, "bsc", 0.02, 0.8)
    ofz, _ = O.frozen_set(n, "bsc", 0.02, 0.8)
    x, _ = S.frames(S.WORKLOADS["bsc_p02_n16"], 0, F)
    fv = torch.zeros(F, (1 << n) // 32, dtype=torch.int32, device=DEV)
    P.polar_reveal(fs, F, to_dev_words(x), fv)
    got = words_np(fv)
    for f in range(F):
        assert np.array_equal(S.unpack_bits(got[f], 1 << n), O.reveal(S.unpack_bits(x[f], 1 << n), ofz))


# ------------------------------------------------------------------ min-sum bit-exact
# 32-leaf frozen patterns (bit j = leaf j frozen): the five that the decoder
# handles by compile-time decoders (repetition, 0x177F7FFF, 0x0117177F,
# 0x00010117, single parity), rate 0 and rate 1, and three neighbours that
# take the generic recursion.
PATTERN_BLOCKS = (0x7FFFFFFF, 0x177F7FFF, 0x0117177F, 0x00010117, 0x00000001,
                  0xFFFFFFFF, 0x00000000, 0x00000117, 0x0017177F, 0x077F7FFF)


def random_code(rng, n, kind):
    N = 1 << n
    if kind == "patterns":      # 32-leaf blocks drawn from PATTERN_BLOCKS
        words = rng.choice(np.array(PATTERN_BLOCKS, dtype=np.uint32), max(1, N // 32))
        return S.unpack_bits(words, N).astype(np.uint8)
    if kind == "random":
        fz = (rng.random(N) < 0.5).astype(np.uint8)
    elif kind == "all_frozen":
        fz = np.ones(N, np.uint8)
    elif kind == "all_info":
        fz = np.zeros(N, np.uint8)
    else:   # polar-like: Bhattacharyya set of a BSC
        fz, _ = O.frozen_set(n, "bsc", 0.05, 0.6)
    return fz


def check_minsum(P, n, kind, F, seed, llr_kind="gauss"):
    N = 1 << n
    rng = np.random.default_rng(seed)
    fz = random_code(rng, n, kind)
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    if llr_kind == "gauss":
        L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
    else:   # BSC-like: +-c with many exact ties in g
        L = (np.float32(2.5) * (1 - 2 * (rng.random((F, N)) < 0.1))).astype(np.float32)
    fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
    fvw = np.stack([S.pack_bits(r) for r in fvb])
    xh, uh = gpu_decode(P, fs, L, fvw)
    for f in range(F):
        ou, ox = O.sc_decode(L[f], fz, fvb[f], "minsum")
        assert np.array_equal(S.unpack_bits(xh[f], N), ox), (n, kind, f)
        assert np.array_equal(S.unpack_bits(uh[f], N), ou), (n, kind, f)


@pytest.mark.parametrize("t", [5, 8, 13])
@pytest.mark.parametrize("n", [1, 2, 4, 5, 6, 9, 12, 15])
@pytest.mark.parametrize("kind", ["random", "polar", "all_info", "all_frozen"])
def test_minsum_bitexact_small(P, n, kind, t):
    P.polar_config_set("subtree_log2", t)
    check_minsum(P, n, kind, F=3, seed=1000 * n + t, llr_kind="gauss")
    check_minsum(P, n, kind, F=2, seed=1000 * n + t + 7, llr_kind="bsc")


@pytest.mark.parametrize("t", [5, 9, 13])
def test_minsum_frozen_pattern_decoders(P, t):
    """Codes built from the 32-leaf patterns with compile-time decoders, with
    Gaussian LLRs and with BSC-like +-c LLRs (exact zeros in g, which the
    rate-1 children inside those patterns must handle): x_hat and u_hat
    bit-exact against the oracle."""
    P.polar_config_set("subtree_log2", t)
    check_minsum(P, 14, "patterns", F=3, seed=4100 + t, llr_kind="gauss")
    check_minsum(P, 14, "patterns", F=3, seed=4200 + t, llr_kind="bsc")


@pytest.mark.parametrize("mode", ["no_shortcuts", "no_graphs", "plain", "no_fuse", "no_pdl",
                                  "prologue", "prologue_no_fuse"])
def test_minsum_bitexact_modes(P, mode):
    if mode.startswith("prologue"):
        P.polar_config_set("prologue", 1)
        P.polar_config_set("fuse", 0 if mode.endswith("no_fuse") else 1)
    elif mode == "no_pdl":
        P.polar_config_set("pdl", 0)
    elif mode == "no_fuse":
        P.polar_config_set("fuse", 0)
    elif mode == "no_shortcuts":
        P.polar_config_set("shortcuts", 0)
    elif mode == "no_graphs":
        P.polar_config_set("graphs", 0)
    else:
        P.polar_config_set("plain", 1)
    P.polar_config_set("subtree_log2", 9)
    for n, kind in ((12, "polar"), (14, "random"), (11, "all_info")):
        check_minsum(P, n, kind, F=3, seed=77 + n, llr_kind="bsc")


def test_batch_of_mixed_frames(P):
    """polar_sc_decode_batch with frames of several lengths and codes."""
    rng = np.random.default_rng(5)
    frames, expect = [], []
    for n in (10, 12, 12, 16, 10):
        N = 1 << n
        fz = random_code(rng, n, "polar")
        fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
        L = rng.normal(0.5, 2.0, N).astype(np.float32)
        fvb = (rng.integers(0, 2, N) * fz).astype(np.uint8)
        llr = torch.from_numpy(L).to(DEV)
        fv = to_dev_words(S.pack_bits(fvb))
        xh = torch.zeros_like(fv)
        frames.append((fs, llr, fv, xh, None))
        expect.append(O.sc_decode(L, fz, fvb, "minsum")[1])
    P.polar_sc_decode_batch(frames)
    torch.cuda.synchronize()
    for (fs, _, _, xh, _), ox in zip(frames, expect):
        assert np.array_equal(S.unpack_bits(words_np(xh), fs.N), ox)


def decode_workload_gpu(P, w, first, count, fkind="minsum", prec="fp32"):
    fs = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    x, y = S.frames(w, first, count)
    xd = to_dev_words(x)
    fv = torch.empty_like(xd)
    P.polar_reveal(fs, count, xd, fv)
    llr = torch.empty(count, w.N, dtype=torch.float32, device=DEV)
    if w.channel == "bsc":
        P.polar_llr_from_channel("bsc", w.param, to_dev_words(y), llr)
    else:
        P.polar_llr_from_channel("biawgn", w.param, torch.from_numpy(y).to(DEV), llr)
    xh = torch.zeros_like(xd)
    uh = torch.zeros_like(xd)
    P.polar_sc_decode_many(fs, count, llr, fv, xh, uh, fkind, prec)
    torch.cuda.synchronize()
    return fs, x, y, words_np(xh), words_np(uh)


@pytest.mark.parametrize("name,check", [("bsc_p02_n16", 100), ("bsc_p03_n20", 16)])
def test_workload_minsum_bitexact(P, name, check):
    w = S.WORKLOADS[name]
    fs, x, y, xh, uh = decode_workload_gpu(P, w, 0, w.frames)
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    assert np.array_equal(S.unpack_bits(fs.mask(), w.N), ofz)
    for f in range(check):
        ou, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "minsum", 32)
        assert np.array_equal(S.unpack_bits(xh[f], w.N), ox), f
        assert np.array_equal(S.unpack_bits(uh[f], w.N), ou), f


def test_workload_biawgn_2_24_sampled(P):
    """Full-size BI-AWGN workload (16 frames of 2^24) decoded together; four
    frames compared element by element with the float32 min-sum oracle."""
    w = S.WORKLOADS["biawgn_s1_n24"]
    fs, x, y, xh, uh = decode_workload_gpu(P, w, 0, w.frames)
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    assert np.array_equal(S.unpack_bits(fs.mask(), w.N), ofz)
    for f in (0, 5, 10, 15):
        ou, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "minsum", 32)
        assert np.array_equal(S.unpack_bits(xh[f], w.N), ox), f


# ------------------------------------------------------------------ exact f, statistics
def test_exact_f_fer_matches_float64_oracle(P):
    """Exact-f FP32 on the GPU vs exact-f FP64 oracle on the same frames:
    FERs within two binomial standard errors, and bit error rates within two
    standard errors of the mean of the per-frame bit error rates (bits of a
    frame fail together, so frames are the independent samples)
    (BI-AWGN sigma^2 = 1, N = 2^12, rate chosen so that the FER sits
    mid-range)."""
    w = S.Workload("fer_biawgn_n12", "biawgn", 1.0, 12, 0.40, 400, 0x5EED + 40)
    fs, x, y, xh, _ = decode_workload_gpu(P, w, 0, w.frames, fkind="exact")
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    g_err = o_err = 0
    g_ber, o_ber = [], []
    for f in range(w.frames):
        xb = S.unpack_bits(x[f], w.N)
        gx = S.unpack_bits(xh[f], w.N)
        g_err += int(not np.array_equal(gx, xb))
        _, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "exact", 64)
        o_err += int(not np.array_equal(ox, xb))
        g_ber.append(float(np.mean(gx != xb)))
        o_ber.append(float(np.mean(ox != xb)))
    T = w.frames
    pg, po = g_err / T, o_err / T
    se = math.sqrt(max(pg * (1 - pg), 1.0 / T) / T + max(po * (1 - po), 1.0 / T) / T)
    assert 0.02 < po < 0.98, po
    assert abs(pg - po) <= 2 * se, (pg, po, se)
    bg, bo = np.mean(g_ber), np.mean(o_ber)
    se_b = math.sqrt(np.var(g_ber) / T + np.var(o_ber) / T)
    assert bo > 0 and abs(bg - bo) <= 2 * se_b, (bg, bo, se_b)


# ------------------------------------------------------------------ reduced storage
def check_store(P, n, kind, F, seed, prec, llr_kind="gauss"):
    N = 1 << n
    rng = np.random.default_rng(seed)
    fz = random_code(rng, n, kind)
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    if llr_kind == "gauss":
        L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
    else:
        L = (np.float32(2.5) * (1 - 2 * (rng.random((F, N)) < 0.1))).astype(np.float32)
    fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
    fvw = np.stack([S.pack_bits(r) for r in fvb])
    xh, uh = gpu_decode(P, fs, L, fvw, "minsum", prec)
    t = min(n, P.polar_config_get("subtree_log2"))      # levels below t stay on chip in float
    for f in range(F):
        sc = O.int8_scale(L[f], P.polar_config_get("int8_target")) if prec == "int8" else 1.0
        ou, ox = O.sc_decode_store(L[f], fz, fvb[f], "minsum", prec, sc, min_level=t)
        assert np.array_equal(S.unpack_bits(xh[f], N), ox), (n, kind, prec, f)
        assert np.array_equal(S.unpack_bits(uh[f], N), ou), (n, kind, prec, f)


@pytest.mark.parametrize("prec", ["fp16", "int8"])
@pytest.mark.parametrize("t", [5, 9, 13])
@pytest.mark.parametrize("n", [3, 5, 8, 12, 15])
def test_reduced_storage_minsum_bitexact(P, prec, t, n):
    """FP16 / INT8 storage: every LLR stored in bulk memory (the channel LLRs on
    entry and the levels >= t) is rounded and saturated exactly as the
    oracle's storage model does, so min-sum decisions match bit for bit."""
    P.polar_config_set("subtree_log2", t)
    check_store(P, n, "polar", 3, 500 + n + t, prec, "gauss")
    check_store(P, n, "random", 2, 600 + n + t, prec, "bsc")


@pytest.mark.parametrize("prec", ["fp16", "int8"])
def test_reduced_storage_workload_bitexact(P, prec):
    w = S.WORKLOADS["bsc_p03_n20"]
    fs, x, y, xh, uh = decode_workload_gpu(P, w, 0, 8, "minsum", prec)
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    for f in range(8):
        L = O.llr_bsc(S.unpack_bits(y[f], w.N), w.param, 32)
        fv = O.reveal(S.unpack_bits(x[f], w.N), ofz)
        sc = O.int8_scale(L, P.polar_config_get("int8_target")) if prec == "int8" else 1.0
        t = min(w.log2n, P.polar_config_get("subtree_log2"))
        ou, ox = O.sc_decode_store(L, ofz, fv, "minsum", prec, sc, min_level=t)
        assert np.array_equal(S.unpack_bits(xh[f], w.N), ox), f


@pytest.mark.parametrize("fkind", ["minsum", "exact"])
def test_subtree_taking_its_parent_step_changes_no_bit(P, fkind):
    """The subtree kernel computing its input's f / g from level t + 1 gives
    the same x_hat / u_hat as the separate streamed step (float32)."""
    rng = np.random.default_rng(41)
    n, F, N = 16, 6, 1 << 16
    fz = random_code(rng, n, "polar")
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
    fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
    fvw = np.stack([S.pack_bits(r) for r in fvb])
    P.polar_config_set("autotune", 0)
    try:
        out = {}
        for t in (9, 13):
            for pro in (0, 1):
                P.polar_config_set("subtree_log2", t)
                P.polar_config_set("prologue", pro)
                out[(t, pro)] = gpu_decode(P, fs, L, fvw, fkind)
        for t in (9, 13):
            assert np.array_equal(out[(t, 0)][0], out[(t, 1)][0])
            assert np.array_equal(out[(t, 0)][1], out[(t, 1)][1])
    finally:
        P.polar_config_set("autotune", 1)


@pytest.mark.parametrize("kind", ["polar", "random", "all_info", "patterns"])
def test_exact_f_same_bits_on_every_path(P, kind):
    """Every decoder path forms the same exact-f float32 values: the plain
    decoder (lane-parallel through shared memory down to single leaves), the
    register tiles with the 32-leaf decoder (top levels lane-parallel, lower
    ones redundant in every lane) at several subtree sizes, and the persistent
    decoder.  x_hat / u_hat agree bit for bit."""
    rng = np.random.default_rng(67)
    n, F, N = 15, 4, 1 << 15
    fz = random_code(rng, n, kind)
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
    fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
    fvw = np.stack([S.pack_bits(r) for r in fvb])
    P.polar_config_set("autotune", 0)
    try:
        P.polar_config_set("plain", 1)
        P.polar_config_set("subtree_log2", 9)
        ref = gpu_decode(P, fs, L, fvw, "exact")
        P.polar_config_set("plain", 0)
        for t in (5, 9, 13):
            P.polar_config_set("subtree_log2", t)
            got = gpu_decode(P, fs, L, fvw, "exact")
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), t
    finally:
        P.polar_config_set("autotune", 1)
    llr = torch.from_numpy(L).to(DEV)
    fv = to_dev_words(fvw)
    xh, uh = torch.full_like(fv, -1), torch.full_like(fv, -1)
    P.polar_sc_decode_persistent([(fs, llr[f], fv[f], xh[f], uh[f]) for f in range(F)],
                                 fkind="exact")
    torch.cuda.synchronize()
    assert np.array_equal(words_np(xh), ref[0]) and np.array_equal(words_np(uh), ref[1])


def test_autotune_picks_a_schedule_and_keeps_results(P):
    w = S.Workload("tune", "bsc", 0.03, 16, 0.7, 8, 0x5EED + 50)
    fs = P.polar_build_frozen_set(w.log2n, w.channel, w.param, w.rate)
    x, y = S.frames(w, 0, w.frames)
    xd = to_dev_words(x)
    fv = torch.empty_like(xd)
    P.polar_reveal(fs, w.frames, xd, fv)
    llr = torch.empty(w.frames, w.N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel("bsc", w.param, to_dev_words(y), llr)
    xh = torch.zeros_like(xd)
    P.polar_tune_clear()
    t, fuse, ms = P.polar_autotune(fs, w.frames, llr, fv, xh)
    split = (fuse >> 8) & 0xFF          # node-unit level, 0 = none
    assert t in (12, 13, 14) and (fuse & 0xFF) in (0, 1, 2, 3) and ms > 0
    assert split == 0 or t < split <= min(w.log2n - 1, t + 4)
    assert fuse >> 16 == 0
    xh2 = torch.zeros_like(xd)
    P.polar_sc_decode_many(fs, w.frames, llr, fv, xh2)       # uses the tuned schedule
    torch.cuda.synchronize()
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    got = words_np(xh2)
    for f in range(w.frames):
        _, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "minsum", 32)
        assert np.array_equal(S.unpack_bits(got[f], w.N), ox)
    assert torch.equal(xh, xh2)
    P.polar_tune_clear()


def test_table1_largest_code_2_27_sampled(P):
    """Table 1's longest code: N = 2^27 on the BI-AWGN channel at SNR 0.161
    (sigma^2 = 1 / 0.161), rate 0.10 (GA set).  Two frames decoded together,
    the first compared element by element with the float32 min-sum oracle."""
    n, s2, R = 27, 1.0 / 0.161, 0.10
    N = 1 << n
    fs = P.polar_build_frozen_set(n, "biawgn", s2, R)
    ofz, K = O.frozen_set(n, "biawgn", s2, R)
    assert fs.K == K and np.array_equal(S.unpack_bits(fs.mask(), N), ofz)
    xs, ys = zip(*[S.device_frame("biawgn", s2, N, 0x7AB1E + 27, i, DEV) for i in range(2)])
    x, y = torch.stack(xs), torch.stack(ys)
    del xs, ys
    fv = torch.empty_like(x)
    P.polar_reveal(fs, 2, x, fv)
    llr = torch.empty(2, N, dtype=torch.float32, device=DEV)
    P.polar_llr_from_channel("biawgn", s2, y, llr)
    xh = torch.full_like(x, -1)
    P.polar_sc_decode_many(fs, 2, llr, fv, xh, None, "minsum", "fp32")
    torch.cuda.synchronize()
    L0 = llr[0].cpu().numpy()
    fvb = S.unpack_bits(words_np(fv[0]), N)
    _, ox = O.sc_decode(L0, ofz, fvb, "minsum")
    assert np.array_equal(S.unpack_bits(words_np(xh[0]), N), ox)


# ------------------------------------------------------------------ verification hash
def _hash_reference(words, key):
    """The frame hash by its definition, with Python integers."""
    M64, P61 = 2 ** 64 - 1, 2 ** 61 - 1
    h = 0
    for i, w in enumerate(words):
        z = (key + (i + 1) * 0x9E3779B97F4A7C15) & M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        z ^= z >> 31
        z = (z & P61) + (z >> 61)
        if z >= P61:
            z -= P61
        h = (h + int(w) * z) % P61
    return h


@pytest.mark.parametrize("n", [3, 5, 12, 16])
def test_frame_hash_matches_definition_and_detects_errors(P, n):
    N, F, key = 1 << n, 4, 0x1234_5678_9ABC_DEF0
    rng = np.random.default_rng(n)
    bits = rng.integers(0, 2, (F, N)).astype(np.uint8)
    bits[1] = bits[0]                                   # identical frames
    bits[2] = bits[0]
    bits[2][N // 3] ^= 1                                # one flipped bit
    words = np.stack([S.pack_bits(r) for r in bits])
    out = torch.zeros(F, dtype=torch.int64, device=DEV)
    P.polar_frame_hash(n, F, to_dev_words(words), key, out)
    torch.cuda.synchronize()
    got = [int(v) & (2 ** 64 - 1) for v in out.cpu().numpy()]
    assert got == [_hash_reference(w, key) for w in words]
    assert got[0] == got[1] and got[0] != got[2]


# ------------------------------------------------------------------ node units
@pytest.mark.parametrize("fkind,prec", [("minsum", "fp32"), ("exact", "fp32"),
                                        ("minsum", "fp16"), ("exact", "fp16"),
                                        ("minsum", "int8"), ("exact", "int8")])
def test_node_units_same_bits(P, fkind, prec):
    """Nodes of 2^s leaves decoded by one CTA per frame (the levels s..t+1
    inside the CTA) give the same x_hat and u_hat, bit for bit, as the
    schedule that streams those levels; min-sum float32 also equals the
    oracle.  Several (N, t, s) shapes and code shapes, fused and unfused
    steps above s, with and without u_hat."""
    rng = np.random.default_rng(91)
    P.polar_config_set("autotune", 0)
    cases = [(12, 5, 7, "random"), (15, 9, 12, "polar"), (15, 9, 10, "polar"),
             (16, 13, 15, "polar"), (14, 8, 13, "all_info"), (13, 6, 9, "all_frozen"),
             (17, 9, 11, "random")]
    for n, t, sp, kind in cases:
        N, F = 1 << n, 3
        fz = random_code(rng, n, kind)
        fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
        if kind == "random" and fkind == "minsum":     # BSC-like: many exact ties in g
            L = (np.float32(2.5) * (1 - 2 * (rng.random((F, N)) < 0.1))).astype(np.float32)
        else:
            L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
        fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
        fvw = np.stack([S.pack_bits(r) for r in fvb])
        P.polar_config_set("subtree_log2", t)
        for fuse in (1, 0):
            P.polar_config_set("fuse", fuse)
            P.polar_config_set("split_log2", 0)
            ref = gpu_decode(P, fs, L, fvw, fkind, prec)
            P.polar_config_set("split_log2", sp)
            got = gpu_decode(P, fs, L, fvw, fkind, prec)
            assert np.array_equal(got[0], ref[0]), (n, t, sp, kind, fuse)
            assert np.array_equal(got[1], ref[1]), (n, t, sp, kind, fuse)
            got_x, _ = gpu_decode(P, fs, L, fvw, fkind, prec, uhat=False)
            assert np.array_equal(got_x, ref[0]), (n, t, sp, kind, fuse)
        if fkind == "minsum" and prec == "fp32":
            for f in range(F):
                ou, ox = O.sc_decode(L[f], fz, fvb[f], "minsum")
                assert np.array_equal(S.unpack_bits(got[0][f], N), ox)
                assert np.array_equal(S.unpack_bits(got[1][f], N), ou)


def test_node_units_on_the_bench_workload(P):
    """The 2^20 workload (16 of its 64 frames) with node units of 2^17 leaves
    at t = 14: bit-exact against the oracle's float32 min-sum."""
    w = S.WORKLOADS["bsc_p03_n20"]
    P.polar_config_set("autotune", 0)
    P.polar_config_set("subtree_log2", 14)
    P.polar_config_set("split_log2", 17)
    fs, x, y, xh, uh = decode_workload_gpu(P, w, 0, 16)
    ofz, _ = O.frozen_set(w.log2n, w.channel, w.param, w.rate)
    for f in range(0, 16, 3):
        ou, ox, _ = O.decode_frame(w.channel, w.param, x[f], y[f], ofz, "minsum", 32)
        assert np.array_equal(S.unpack_bits(xh[f], w.N), ox)
        assert np.array_equal(S.unpack_bits(uh[f], w.N), ou)
