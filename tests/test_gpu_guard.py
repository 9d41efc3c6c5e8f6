"""Guard mode: no kernel writes outside its scratch or its output buffers.

compute-sanitizer is not available, so out-of-range global writes are caught
the way a guard-page allocator catches them: in guard mode the library's
scratch workspaces carry zones of a fixed byte pattern on both sides, checked
after every decode call (POLAR_EFAULT if a byte changed), and the tests below
surround the caller's buffers with zones of their own.  Every decode path runs
in guard mode with its results compared bit for bit with the unguarded run;
a zone spoiled on purpose (a write inside the allocation) must be reported.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402

DEV = "cuda:0"
MARGIN = 4096          # int32 words of canary on each side of a caller's buffer
CANARY = 0x5A5A5A5A


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


KEYS = ("guard", "subtree_log2", "shortcuts", "graphs", "plain", "fuse", "prologue",
        "autotune", "persist_log2", "split_log2")


@pytest.fixture(autouse=True)
def restore_config(P):
    saved = {k: P.polar_config_get(k) for k in KEYS}
    yield
    for k, v in saved.items():
        P.polar_config_set(k, v)


def fenced(n_words, fill, dtype=torch.int32):
    """A device buffer of n_words with MARGIN canary words on either side;
    returns (whole, view)."""
    whole = torch.full((n_words + 2 * MARGIN,), CANARY, dtype=torch.int32, device=DEV)
    view = whole[MARGIN:MARGIN + n_words]
    if dtype == torch.float32:
        view = view.view(torch.float32)
    view.fill_(fill)
    return whole, view


def fences_intact(whole):
    h = whole.cpu()
    return bool((h[:MARGIN] == CANARY).all()) and bool((h[-MARGIN:] == CANARY).all())


def problem(seed, n, F, kind="polar"):
    rng = np.random.default_rng(seed)
    N = 1 << n
    if kind == "polar":
        fz, _ = O.frozen_set(n, "bsc", 0.05, 0.6)
    else:
        fz = (rng.random(N) < 0.5).astype(np.uint8)
    L = rng.normal(0.5, 2.0, (F, N)).astype(np.float32)
    fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
    return fz, L, fvb


def decode_fenced(P, fs, L, fvb, fkind="minsum", prec="fp32"):
    """Decode with every caller buffer fenced; returns (x_hat, u_hat) words
    and checks that the fences and the inputs are untouched."""
    F, N = L.shape
    W = max(N // 32, 1)
    lw, llr = fenced(F * N, 0.0, torch.float32)
    llr.copy_(torch.from_numpy(L.reshape(-1)).to(DEV))
    fw, fv = fenced(F * W, 0)
    fv.copy_(torch.from_numpy(np.stack([S.pack_bits(r) for r in fvb]).reshape(-1).view(np.int32))
             .to(DEV))
    xw, xh = fenced(F * W, -1)
    uw, uh = fenced(F * W, -1)
    llr_before, fv_before = llr.clone(), fv.clone()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()            # a non-default stream: graph replay is allowed
    P.polar_sc_decode_many(fs, F, llr, fv, xh, uh, fkind, prec, stream)
    stream.synchronize()
    for w in (lw, fw, xw, uw):
        assert fences_intact(w)
    assert torch.equal(llr, llr_before) and torch.equal(fv, fv_before)
    return xh.view(F, W).cpu().numpy().view(np.uint32), uh.view(F, W).cpu().numpy().view(np.uint32)


MODES = {
    "graphs_t13": {"subtree_log2": 13},
    "graphs_t9": {"subtree_log2": 9},
    "t5": {"subtree_log2": 5},
    "no_graphs_t9": {"subtree_log2": 9, "graphs": 0},
    "no_shortcuts_t9": {"subtree_log2": 9, "shortcuts": 0},
    "unfused_t9": {"subtree_log2": 9, "fuse": 0},
    "prologue_t9": {"subtree_log2": 9, "prologue": 1},
    "plain": {"plain": 1, "subtree_log2": 9},
    "nodes_t9_s12": {"subtree_log2": 9, "split_log2": 12},
    "nodes_t9_s10_unfused": {"subtree_log2": 9, "split_log2": 10, "fuse": 0},
    "nodes_t13_s14": {"subtree_log2": 13, "split_log2": 14},
}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("fkind,prec", [("minsum", "fp32"), ("exact", "fp32"),
                                        ("minsum", "fp16"), ("minsum", "int8")])
def test_every_launched_path_stays_inside_its_buffers(P, mode, fkind, prec):
    if mode in ("plain", "prologue_t9") and prec != "fp32":
        pytest.skip("plain and prologue schedules are float32 paths")
    n, F = 15, 3
    fz, L, fvb = problem(101, n, F, "random" if mode == "t5" else "polar")
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    P.polar_config_set("autotune", 0)
    for k, v in MODES[mode].items():
        P.polar_config_set(k, v)
    P.polar_config_set("guard", 0)
    ref = decode_fenced(P, fs, L, fvb, fkind, prec)
    P.polar_config_set("guard", 1)
    got = decode_fenced(P, fs, L, fvb, fkind, prec)     # raises on POLAR_EFAULT
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    if fkind == "minsum" and prec == "fp32":
        for f in range(F):
            ou, ox = O.sc_decode(L[f], fz, fvb[f], "minsum")
            assert np.array_equal(S.unpack_bits(got[0][f], 1 << n), ox)


def test_persistent_and_batch_paths_stay_inside_their_buffers(P):
    P.polar_config_set("guard", 1)
    P.polar_config_set("persist_log2", 9)
    frames, fences, expect = [], [], []
    for i, n in enumerate((16, 12, 14, 10, 15)):
        fz, L, fvb = problem(200 + i, n, 1)
        fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
        N, W = 1 << n, max((1 << n) // 32, 1)
        lw, llr = fenced(N, 0.0, torch.float32)
        llr.copy_(torch.from_numpy(L[0]).to(DEV))
        fw, fv = fenced(W, 0)
        fv.copy_(torch.from_numpy(S.pack_bits(fvb[0]).view(np.int32)).to(DEV))
        xw, xh = fenced(W, -1)
        uw, uh = fenced(W, -1)
        frames.append((fs, llr, fv, xh, uh))
        fences += [lw, fw, xw, uw]
        expect.append(O.sc_decode(L[0], fz, fvb[0], "minsum"))
    for call in ("persistent", "batch"):
        for f in frames:
            f[3].fill_(-1)
            f[4].fill_(-1)
        if call == "persistent":
            P.polar_sc_decode_persistent(frames)
        else:
            P.polar_sc_decode_batch(frames)
        torch.cuda.synchronize()
        assert all(fences_intact(w) for w in fences), call
        for (fs, _, _, xh, uh), (ou, ox) in zip(frames, expect):
            N = fs.N
            assert np.array_equal(S.unpack_bits(xh.cpu().numpy().view(np.uint32), N), ox), call
            assert np.array_equal(S.unpack_bits(uh.cpu().numpy().view(np.uint32), N), ou), call


def test_a_spoiled_guard_zone_is_reported(P):
    """Positive control: the checker reports a changed guard byte, and the
    next decode (zone restored) passes."""
    P.polar_config_set("guard", 1)
    P.polar_config_set("autotune", 0)
    P.polar_config_set("subtree_log2", 9)
    n, F = 14, 2
    fz, L, fvb = problem(303, n, F)
    fs = P.polar_frozen_set_from_mask(n, S.pack_bits(fz))
    stream = torch.cuda.Stream()
    llr = torch.from_numpy(L).to(DEV)
    fv = torch.from_numpy(np.stack([S.pack_bits(r) for r in fvb]).view(np.int32)).to(DEV)
    xh = torch.zeros_like(fv)
    torch.cuda.synchronize()
    P.polar_sc_decode_many(fs, F, llr, fv, xh, None, "minsum", "fp32", stream)
    P.polar_debug_spoil_guard(stream)
    with pytest.raises(P.PolarError) as e:
        P.polar_sc_decode_many(fs, F, llr, fv, xh, None, "minsum", "fp32", stream)
    assert e.value.status == P.POLAR_EFAULT
    P.polar_sc_decode_many(fs, F, llr, fv, xh, None, "minsum", "fp32", stream)
    stream.synchronize()
