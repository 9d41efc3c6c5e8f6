"""CPU checks of the C ABI: the library builds, loads, exports every function
declared in include/*.h, and rejects bad arguments on the host before any
CUDA call; host-side construction equals the oracle's."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(polar_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (polar_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(P.lib(), n)


def test_library_is_built_for_sm_103a(P):
    log = open(os.path.join(os.path.dirname(P.LIB_PATH), "subtree.cu.log")).read()
    assert "arch=compute_103a,code=sm_103a" in log


def test_strerror_and_config(P):
    assert P.lib().polar_strerror(-1).decode() == "invalid argument"
    old = P.polar_config_get("subtree_log2")
    P.polar_config_set("subtree_log2", 9)
    assert P.polar_config_get("subtree_log2") == 9
    P.polar_config_set("subtree_log2", old)
    with pytest.raises(P.PolarError):
        P.polar_config_set("subtree_log2", 40)
    with pytest.raises(P.PolarError):
        P.polar_config_set("no_such_key", 1)
    assert P.polar_config_get("persistent") == 1
    assert P.polar_config_get("persist_log2") == 13
    with pytest.raises(P.PolarError):
        P.polar_config_set("persist_log2", 4)
    with pytest.raises(P.PolarError):
        P.polar_config_set("persistent", 3)
    assert P.polar_config_get("guard") == 0
    P.polar_config_set("guard", 1)
    assert P.polar_config_get("guard") == 1
    P.polar_config_set("guard", 0)
    assert P.lib().polar_strerror(P.POLAR_EFAULT).decode().startswith("out-of-range write")


def test_argument_errors_are_host_side(P):
    L = P.lib()
    fs = P.polar_build_frozen_set(10, "bsc", 0.03, 0.5)
    # null device pointers / bad enums / bad counts: rejected before any CUDA call
    assert L.polar_sc_decode_many(fs.handle, 1, None, None, None, None, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_many(fs.handle, 0, 16, 16, 16, None, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_many(fs.handle, 1, 16, 16, 16, None, 7, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_many(fs.handle, 1, 16, 16, 16, None, 0, 9, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_many(fs.handle, 1, 18, 16, 16, None, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_many(None, 1, 16, 16, 16, None, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_llr_from_channel(0, 0.7, 16, 1, 16, 64, None) == P.POLAR_EINVAL
    assert L.polar_llr_from_channel(0, 0.1, 16, 0, 16, 64, None) == P.POLAR_EINVAL
    assert L.polar_llr_from_channel(0, 0.1, 16, 1, 16, 33, None) == P.POLAR_EINVAL
    assert L.polar_llr_from_channel(1, -1.0, 16, 0, 16, 64, None) == P.POLAR_EINVAL
    assert L.polar_llr_from_channel(1, 1.0, 16, 0, 16, 0, None) == P.POLAR_OK   # empty
    assert L.polar_encode(0, 1, 16, 16, None) == P.POLAR_EINVAL
    assert L.polar_encode(28, 1, 16, 16, None) == P.POLAR_EINVAL
    # verification hash: sizes, null and misaligned pointers; key-rate formula
    assert L.polar_frame_hash(0, 1, 16, 1, 16, None) == P.POLAR_EINVAL
    assert L.polar_frame_hash(10, 1, None, 1, 16, None) == P.POLAR_EINVAL
    assert L.polar_frame_hash(10, 1, 16, 1, 12, None) == P.POLAR_EINVAL
    assert P.polar_key_rate(0.5, 0.1, 0.9, 0.8, 0.3) == pytest.approx(0.5 * 0.9 * (0.9 * 0.8 - 0.3))
    # persistent decoder: empty queue, null table, unknown storage
    desc = (P.FrameDesc * 1)(P.FrameDesc(fs.handle.value, 16, 16, 16, None))
    assert L.polar_sc_decode_persistent(0, desc, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_persistent(1, None, 0, 0, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_persistent(1, desc, 0, 3, None) == P.POLAR_EINVAL
    assert L.polar_sc_decode_persistent(1, desc, 0, -1, None) == P.POLAR_EINVAL
    bad = (P.FrameDesc * 1)(P.FrameDesc(fs.handle.value, 20, 16, 16, None))   # llr not 16-B
    assert L.polar_sc_decode_persistent(1, bad, 0, 0, None) == P.POLAR_EINVAL
    with pytest.raises(P.PolarError):
        P.polar_build_frozen_set(10, "bsc", 0.7, 0.5)
    with pytest.raises(P.PolarError):
        P.polar_build_frozen_set(0, "bsc", 0.1, 0.5)
    with pytest.raises(P.PolarError):
        P.polar_build_frozen_set(10, "biawgn", 1.0, 1.5)


@pytest.mark.parametrize("case", [(10, "bsc", 0.02, 0.8), (16, "bsc", 0.02, 0.80),
                                  (20, "bsc", 0.03, 0.75), (12, "biawgn", 1.0, 0.44),
                                  (18, "biawgn", 1.0, 0.44), (14, "biawgn", 0.5, 0.93),
                                  (1, "bsc", 0.1, 0.5), (4, "biawgn", 2.0, 0.25)])
def test_library_construction_equals_oracle(P, case):
    import oracle as O
    from paper_1204_5882_gb300 import synth as S
    n, ch, par, R = case
    fs = P.polar_build_frozen_set(n, ch, par, R)
    ofz, K = O.frozen_set(n, ch, par, R)
    assert fs.K == K
    assert np.array_equal(S.unpack_bits(fs.mask(), 1 << n), ofz)
    assert fs.sum_pe == pytest.approx(O.fer_bound(n, ch, par, ofz), rel=1e-9)


@pytest.mark.parametrize("case", [(3, "bsc", 0.11, 128, 0.5, 0.0), (10, "bsc", 0.03, 16, 0.75, 0.0),
                                  (12, "bsc", 0.02, 16, 0.0, 0.1), (12, "biawgn", 1.0, 16, 0.44, 0.0),
                                  (14, "biawgn", 0.8, 8, 0.0, 0.05), (16, "bsc", 0.02, 16, 0.0, 0.1)])
def test_library_degraded_construction_equals_oracle(P, case):
    """The library's degraded construction (classes as mass / crossover,
    heap-driven greedy merging) and the oracle's (likelihood pairs, linear
    scans) are separate derivations of Tal and Vardy's method: the same
    frozen sets and K, and the summed bounds within accumulated rounding."""
    import oracle as O
    from paper_1204_5882_gb300 import synth as S
    n, ch, par, mu, rate, smax = case
    fs = P.polar_build_frozen_set_tv(n, ch, par, mu, rate, smax)
    fz, K, spe = O.frozen_set_tv(n, ch, par, rate=rate, sum_pe_max=smax, mu=mu)
    assert fs.K == K
    assert np.array_equal(S.unpack_bits(fs.mask(), 1 << n), fz)
    assert fs.sum_pe == pytest.approx(spe, rel=1e-6, abs=1e-300)
    with pytest.raises(P.PolarError):
        P.polar_build_frozen_set_tv(n, ch, par, 3, rate, smax)


@pytest.mark.parametrize("case", [(12, "biawgn", 1.0, 0.1), (16, "biawgn", 1 / 1.097, 0.1),
                                  (14, "bsc", 0.02, 0.1), (10, "biawgn", 4.0, 0.01)])
def test_library_sum_rule_construction_equals_oracle(P, case):
    import oracle as O
    from paper_1204_5882_gb300 import synth as S
    n, ch, par, smax = case
    fs = P.polar_build_frozen_set_sum(n, ch, par, smax)
    fz, K, spe = O.frozen_set_sum(n, ch, par, smax)
    assert fs.K == K and np.array_equal(S.unpack_bits(fs.mask(), 1 << n), fz)
    assert fs.sum_pe == pytest.approx(spe, rel=1e-9)


def test_frozen_set_from_mask_roundtrip(P):
    m = np.array([0xDEADBEEF, 0x0], dtype=np.uint32)
    fs = P.polar_frozen_set_from_mask(6, m)
    assert np.array_equal(fs.mask(), m)
    assert fs.K == 64 - bin(0xDEADBEEF).count("1")
    fs = P.polar_frozen_set_from_mask(3, np.array([0xFFFFFF0F], dtype=np.uint32))
    assert fs.mask()[0] == 0x0F and fs.K == 4


def test_server_config_rejected_on_host(P):
    import ctypes as C
    h = C.c_void_p()
    for cfg in (P.ServerConfig(0, 0, 16, 1 << 30, 0, 0, 0), P.ServerConfig(0, 4, 0, 1 << 30, 0, 0, 0),
                P.ServerConfig(0, 4, 16, 1 << 30, 5, 0, 0), P.ServerConfig(0, 4, 16, 1 << 30, 0, 7, 0),
                P.ServerConfig(0, 4, 16, 1 << 30, 0, 0, 99),
                P.ServerConfig(-1, 4, 16, 1 << 30, 0, 0, 0),
                P.ServerConfig(0, 4, 16, 1 << 30, 0, 1, 0, 1, 0),      # persistent needs fp32
                P.ServerConfig(0, 4, 16, 1 << 30, 0, 0, 0, 1, 28),     # max_log2n range
                P.ServerConfig(0, 5000, 16, 1 << 30, 0, 0, 0, 1, 0),   # resident CTA cap
                P.ServerConfig(0, 4, 16, 1 << 30, 0, 0, 0, 2, 0)):
        assert P.lib().polar_server_create(C.byref(cfg), C.byref(h)) == P.POLAR_EINVAL
    assert P.lib().polar_server_submit(None, None, None) == P.POLAR_EINVAL
    assert P.lib().polar_server_poll(None, 1, None) == P.POLAR_EINVAL
    assert P.lib().polar_server_cancel(None, 1) == P.POLAR_EINVAL
    assert P.lib().polar_frozen_set_upload(None, 0) == P.POLAR_EINVAL
    fs = P.polar_build_frozen_set(10, "bsc", 0.05, 0.5)
    assert P.lib().polar_frozen_set_upload(fs.handle, -1) == P.POLAR_EINVAL
    assert P.lib().polar_strerror(P.POLAR_ECANCELED).decode() == "cancelled"


def test_tune_table_roundtrip(P, tmp_path):
    src = tmp_path / "tune_in.json"
    src.write_text(
        '{"polar_tune": [\n'
        '  {"device": 0, "log2n": 20, "nframes": 64, "fkind": 0, "prec": 0, '
        '"subtree_log2": 14, "fuse": 1, "ms": 9.5},\n'
        '  {"device": 0, "log2n": 24, "nframes": 16, "fkind": 1, "prec": 1, '
        '"subtree_log2": 13, "fuse": 0, "ms": 100.25}\n]}\n')
    P.polar_tune_clear()
    assert P.polar_tune_load(str(src))
    out = tmp_path / "tune_out.json"
    P.polar_tune_save(str(out))
    text = out.read_text()
    assert '"log2n": 20, "nframes": 64' in text and '"subtree_log2": 14, "fuse": 1' in text
    assert '"log2n": 24, "nframes": 16, "fkind": 1, "prec": 1, "subtree_log2": 13' in text
    assert not P.polar_tune_load(str(tmp_path / "missing.json"))
    P.polar_tune_clear()


def test_log_switch_reports_construction(P):
    """POLAR_LOG=1 prints one line per frozen-set construction on stderr;
    unset or 0, the library prints nothing."""
    import sys
    code = ("from paper_1204_5882_gb300 import polar as P; "
            "P.polar_build_frozen_set(10, 'bsc', 0.05, 0.5)")
    out = {}
    for val in ("1", "0", None):
        env = {k: v for k, v in os.environ.items() if k != "POLAR_LOG"}
        if val is not None:
            env["POLAR_LOG"] = val
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out[val] = r.stderr
    assert "[polar] frozen set (rate): log2n 10, bsc 0.05 -> status 0, K 512" in out["1"]
    assert "[polar]" not in out["0"] and "[polar]" not in out[None]


def _noalloc_need(log2n, nframes, prec_bytes, t=13, int8=False):
    """Bytes the allocation-free decode needs, by the sizing rule its header
    states: mask N/8 and class table N/64 (shortcuts on), each rounded up to
    256, INT8 scales 4 per frame rounded up to 256, levels F (N - 2^t) b."""
    up = lambda v: (v + 255) // 256 * 256  # noqa: E731
    N = 1 << log2n
    return (up(N // 8) + up(N // 64) + (up(4 * nframes) if int8 else 0)
            + nframes * (N - (1 << t)) * prec_bytes)


# (log2 N, frames, bytes per stored LLR, int8) -> fits; the header's examples
# at t = 13 and the next size up of each.
NOALLOC_EXAMPLES = [
    ((20, 3, 4, False), True), ((20, 4, 4, False), False),
    ((21, 1, 4, False), True), ((21, 2, 4, False), False), ((22, 1, 4, False), False),
    ((20, 7, 2, False), True), ((20, 8, 2, False), False),
    ((22, 1, 2, False), True), ((22, 2, 2, False), False),
    ((20, 15, 1, True), True), ((20, 16, 1, True), False),
    ((22, 3, 1, True), True), ((22, 4, 1, True), False),
]


def test_noalloc_documented_capacities(P):
    """Every capacity example in the header of the allocation-free decode
    holds for the array size the library reports, and the header names
    exactly these examples."""
    cap = P.polar_static_scratch_bytes()
    assert cap == 16 << 20
    for (n, F, b, i8), fits in NOALLOC_EXAMPLES:
        assert (_noalloc_need(n, F, b, int8=i8) <= cap) == fits, (n, F, b, i8)
    hdr = open(os.path.join(ROOT, "include", "polar.h")).read()
    doc = hdr[hdr.index("Capacity: the mask"):hdr.index("Larger requests return POLAR_EINVAL")]
    doc = " ".join(doc.replace("*", " ").split())
    for phrase in ("up to 3 frames of 2^20 or 1 frame of 2^21 in FP32",
                   "7 frames of 2^20 or 1 frame of 2^22 in FP16",
                   "15 frames of 2^20 or 3 frames of 2^22 in INT8"):
        assert phrase in doc, phrase
