"""Pins for the oracle's transform, f and SC decoder (CPU only).

Each pin is fixed by mathematics independent of the oracle's own code:
an explicit Kronecker product, closed forms at N = 2, the literal
2 atanh(tanh tanh) form, and brute-force bit-channel likelihoods over all
future bits for N <= 16 (the definition SC evaluates recursively, Sec. 4).
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O


def kron_G(n):
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    for _ in range(n):
        G = np.kron(G, F)
    return G


# ------------------------------------------------------------------ transform
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_encode_matches_kronecker_power(n):
    N = 1 << n
    G = kron_G(n)
    rng = np.random.default_rng(n)
    for _ in range(20):
        u = rng.integers(0, 2, N).astype(np.uint8)
        assert np.array_equal(O.encode(u), (u.astype(np.int64) @ G) % 2)


def test_encode_n2_closed_form():
    for u0, u1 in itertools.product((0, 1), repeat=2):
        assert O.encode([u0, u1]).tolist() == [u0 ^ u1, u1]


@pytest.mark.parametrize("n", [1, 4, 9, 14])
def test_encode_is_involution(n):
    rng = np.random.default_rng(100 + n)
    u = rng.integers(0, 2, 1 << n).astype(np.uint8)
    assert np.array_equal(O.encode(O.encode(u)), u)


# ------------------------------------------------------------------ f and g
def test_f_exact_closed_form_n2():
    """Leaf LLRs at N = 2: L(u0) = ln[(1 + e^{a+b}) / (e^a + e^b)],
    L(u1) = b + (1 - 2 u0) a."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        a, b = rng.normal(0, 4, 2)
        u, x, leaf = O.sc_decode(np.array([a, b]), [0, 0], [0, 0], "exact", leaf=True)
        l0 = math.log1p(math.exp(a + b)) - math.log(math.exp(a) + math.exp(b))
        assert leaf[0] == pytest.approx(l0, rel=1e-12, abs=1e-13)
        assert u[0] == (1 if leaf[0] < 0 else 0)
        assert leaf[1] == b + (1 - 2 * int(u[0])) * a
        assert u[1] == (1 if leaf[1] < 0 else 0)
        assert x.tolist() == [u[0] ^ u[1], u[1]]


def test_f_exact_equals_literal_atanh():
    rng = np.random.default_rng(8)
    for lim, rtol in ((10.0, 1e-10), (15.0, 1e-8)):
        for _ in range(2000):
            a, b = rng.uniform(-lim, lim, 2)
            lit = 2.0 * math.atanh(math.tanh(a / 2) * math.tanh(b / 2))
            assert O.f_exact(a, b) == pytest.approx(lit, rel=rtol, abs=1e-15)


def test_f_exact_float32_close_to_double():
    rng = np.random.default_rng(9)
    for _ in range(2000):
        a, b = (float(v) for v in rng.normal(0, 5, 2).astype(np.float32))
        assert O.f_exact(a, b, 32) == pytest.approx(O.f_exact(a, b), rel=1e-5, abs=1e-6)


def test_f_limits():
    assert O.f_exact(0.0, 3.0) == 0.0
    assert O.f_exact(800.0, 2.5) == pytest.approx(2.5, rel=1e-15)
    assert O.f_exact(-40.0, 40.0) == pytest.approx(-40.0 + math.log(2), rel=1e-12)
    assert O.f_exact(1e-8, 1e-8) == pytest.approx(0.5e-16, rel=1e-6)


def _f_literal(a, b, dps=60):
    """2 atanh(tanh(a/2) tanh(b/2)) evaluated literally in high precision.

    The working precision grows with the inputs so that tanh(x/2) = 1 - 2e^-x
    still differs from 1: the literal definition, with no rearrangement."""
    mpmath = pytest.importorskip("mpmath")
    big = max(abs(a), abs(b))
    with mpmath.workdps(int(dps + big / 2.3)):
        a, b = mpmath.mpf(a), mpmath.mpf(b)
        return float(2 * mpmath.atanh(mpmath.tanh(a / 2) * mpmath.tanh(b / 2)))


@pytest.mark.parametrize("a", [50.0, 700.0, 710.0, 1e4, 1e6])
def test_f_exact_both_inputs_large(a):
    """Both inputs large: f(a, a + d) = a - ln(1 + e^-d) up to e^-(2a+d), and
    finite in both precisions (a form through phi(phi(A) + phi(B)) returns
    +-inf here once phi underflows)."""
    for d in (0.0, 0.25, 1.0, 3.0, 12.0, 40.0):
        want = a - math.log1p(math.exp(-d))
        for sa, sb in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
            got = O.f_exact(sa * a, sb * (a + d))
            assert math.isfinite(got)
            assert got == pytest.approx(sa * sb * want, rel=1e-12)
            g32 = O.f_exact(float(np.float32(sa * a)), float(np.float32(sb * (a + d))), 32)
            assert math.isfinite(g32)
            assert g32 == pytest.approx(sa * sb * want, rel=1e-6)
    if a <= 710.0:
        assert O.f_exact(a, a + 1.0) == pytest.approx(_f_literal(a, a + 1.0), rel=1e-14)


def test_f_exact_all_magnitudes_against_literal():
    """Log-uniform magnitudes from 1e-9 to 1e3, any signs: the double oracle
    keeps relative precision everywhere (tiny results included), the float
    oracle is within float rounding."""
    rng = np.random.default_rng(11)
    for _ in range(600):
        a, b = 10.0 ** rng.uniform(-9, 3, 2) * rng.choice([-1.0, 1.0], 2)
        lit = _f_literal(a, b)
        assert O.f_exact(a, b) == pytest.approx(lit, rel=1e-13)
        a32, b32 = float(np.float32(a)), float(np.float32(b))
        assert O.f_exact(a32, b32, 32) == pytest.approx(_f_literal(a32, b32), rel=2e-5)


def test_f_exact_continuous_across_the_form_switch():
    """Inputs around the magnitude where the evaluation changes form: the
    literal definition decides, to a few ulp."""
    for A in np.linspace(15.5, 16.5, 41):
        for B in (A, A + 0.01, A + 1.0, A + 30.0, 2.0 * A):
            assert O.f_exact(A, B) == pytest.approx(_f_literal(A, B), rel=4e-16 * 8)
            a32, b32 = float(np.float32(A)), float(np.float32(B))
            assert O.f_exact(a32, b32, 32) == pytest.approx(_f_literal(a32, b32), rel=1e-6)


@pytest.mark.parametrize("chan,param,n", [("bsc", 0.02, 16), ("biawgn", 1.0, 18)])
def test_exact_leaf_llrs_finite_on_paper_workloads(chan, param, n):
    """Exact-f SC on a frame shaped like the paper's workloads: every leaf LLR
    is finite in both precisions (large |L| are common deep in the tree)."""
    from paper_1204_5882_gb300 import synth
    N = 1 << n
    w = synth.Workload("t", chan, param, n, 0.8 if chan == "bsc" else 0.44, 1, 0x5EED + 40 + n)
    x, y = synth.frame(w, 0)
    frozen, _ = O.frozen_set(n, chan, param, w.rate)
    xb = synth.unpack_bits(x, N)
    fval = O.reveal(xb, frozen)
    for prec in (64, 32):
        if chan == "bsc":
            L = O.llr_bsc(synth.unpack_bits(y, N), param, prec)
        else:
            L = O.llr_biawgn(y, param, prec)
        _, _, leaf = O.sc_decode(L, frozen, fval, "exact", leaf=True)
        assert np.isfinite(leaf).all()
        assert np.abs(leaf).max() > (100.0 if prec == 32 else 800.0)


def test_f_minsum_closed_form():
    rng = np.random.default_rng(10)
    for _ in range(500):
        a, b = rng.normal(0, 3, 2)
        s = math.copysign(1.0, a) * math.copysign(1.0, b)
        assert O.f_minsum(a, b) == s * min(abs(a), abs(b))


# ------------------------------------------------------------------ brute force
def _codewords(n):
    N = 1 << n
    U = np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.int64)
    return U, (U @ kron_G(n)) % 2


def _random_case(rng, N):
    frozen = rng.integers(0, 2, N).astype(np.uint8)
    if rng.random() < 0.2:
        frozen[:] = 0
    fval = (rng.integers(0, 2, N) * frozen).astype(np.uint8)
    return frozen, fval


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_sc_exact_equals_bruteforce_bit_channel(n):
    """Exact-f SC leaf LLR = ln sum_{future u} prod W(y|x) | u_i=0 minus the
    same with u_i = 1, given the decoder's own past decisions."""
    N = 1 << n
    U, X = _codewords(n)
    rng = np.random.default_rng(20 + n)
    for _ in range(25 if n == 4 else 60):
        L = rng.normal(2.0, 2.0, N) * rng.choice([-1, 1], N)
        frozen, fval = _random_case(rng, N)
        u, x, leaf = O.sc_decode(L, frozen, fval, "exact", leaf=True)
        metric = 0.5 * ((1 - 2 * X) @ L)          # ln prod e^{(1-2x)L/2}
        for i in range(N):
            past = np.all(U[:, :i] == u[:i], axis=1)
            s0 = np.logaddexp.reduce(metric[past & (U[:, i] == 0)])
            s1 = np.logaddexp.reduce(metric[past & (U[:, i] == 1)])
            assert leaf[i] == pytest.approx(s0 - s1, rel=1e-9, abs=1e-9)
            if abs(s0 - s1) > 1e-9:
                want = fval[i] if frozen[i] else int(s0 - s1 < 0)
                assert u[i] == want
        assert np.array_equal(x, O.encode(u))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_sc_minsum_equals_bruteforce_maxlog(n):
    """Min-sum SC is max-log SC: leaf LLR = max corr | u_i=0 - max corr | u_i=1,
    corr = 1/2 sum (1-2x_j) L_j.  Small-integer LLRs make both exact in
    float32, so the comparison is bit-exact, ties (L = 0) included."""
    N = 1 << n
    U, X = _codewords(n)
    rng = np.random.default_rng(40 + n)
    for _ in range(40 if n == 4 else 100):
        L = rng.integers(-4, 5, N).astype(np.float32)
        frozen, fval = _random_case(rng, N)
        u, x, leaf = O.sc_decode(L, frozen, fval, "minsum", leaf=True)
        corr = 0.5 * ((1 - 2 * X) @ L.astype(np.float64))
        for i in range(N):
            past = np.all(U[:, :i] == u[:i], axis=1)
            d = corr[past & (U[:, i] == 0)].max() - corr[past & (U[:, i] == 1)].max()
            assert float(leaf[i]) == d
            want = fval[i] if frozen[i] else int(d < 0)
            assert u[i] == want
        assert np.array_equal(x, O.encode(u))


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("fkind", ["minsum", "exact"])
@pytest.mark.parametrize("n", [1, 5, 10, 12])
def test_rate_one_is_hard_decision(fkind, n):
    N = 1 << n
    rng = np.random.default_rng(60 + n)
    L = rng.normal(0, 3, N).astype(np.float32)
    L[L == 0] = 1.0
    if fkind == "exact":
        # Exact f shrinks products of tanh's: keep |L| large enough that no
        # leaf LLR underflows to a tie in float64 (the identity is exact only
        # while every f stays non-zero).
        L = (np.sign(L) * (6.0 + np.abs(L))).astype(np.float64)
    z = np.zeros(N, np.uint8)
    _, x = O.sc_decode(L, z, z, fkind)
    assert np.array_equal(x, (L < 0).astype(np.uint8))


@pytest.mark.parametrize("n", [1, 6, 11])
def test_rate_zero_returns_encoded_frozen_values(n):
    N = 1 << n
    rng = np.random.default_rng(70 + n)
    L = rng.normal(0, 3, N).astype(np.float32)
    ones = np.ones(N, np.uint8)
    fval = rng.integers(0, 2, N).astype(np.uint8)
    u, x = O.sc_decode(L, ones, fval, "minsum")
    assert np.array_equal(u, fval)
    assert np.array_equal(x, O.encode(fval))


@pytest.mark.parametrize("fkind", ["minsum", "exact"])
def test_noise_free_channel_decodes_exactly(fkind):
    n = 12
    N = 1 << n
    rng = np.random.default_rng(80)
    for rate in (0.3, 0.9, 1.0):
        frozen = (rng.random(N) > rate).astype(np.uint8)
        x = rng.integers(0, 2, N).astype(np.uint8)
        fv = O.reveal(x, frozen)
        # Strong channels for exact f: products of 4096 tanh's must not
        # underflow to a tie (the claim holds in exact arithmetic).
        p, s2 = (0.05, 0.8) if fkind == "minsum" else (1e-4, 0.1)
        for L in (O.llr_bsc(x, p), O.llr_biawgn(1.0 - 2.0 * x, s2, 64)):
            u, xh = O.sc_decode(L, frozen, fv, fkind)
            assert np.array_equal(xh, x)


def test_minsum_decisions_scale_invariant():
    n = 12
    N = 1 << n
    rng = np.random.default_rng(90)
    frozen = (rng.random(N) < 0.4).astype(np.uint8)
    fval = (rng.integers(0, 2, N) * frozen).astype(np.uint8)
    L = rng.normal(1.0, 2.0, N).astype(np.float32)
    _, x0 = O.sc_decode(L, frozen, fval, "minsum")
    for k in (-3, 1, 5):
        _, xk = O.sc_decode((L * np.float32(2.0 ** k)).astype(np.float32), frozen, fval, "minsum")
        assert np.array_equal(x0, xk)


@pytest.mark.parametrize("fkind", ["minsum", "exact"])
def test_codeword_sign_symmetry(fkind):
    """Flipping the LLRs by a codeword c (c = v F^n with v zero on the frozen
    set) flips x_hat by c, on tie-free inputs."""
    n = 11
    N = 1 << n
    rng = np.random.default_rng(95)
    frozen = (rng.random(N) < 0.5).astype(np.uint8)
    fval = (rng.integers(0, 2, N) * frozen).astype(np.uint8)
    L = rng.normal(0.5, 2.0, N)
    if fkind == "exact":   # keep every f away from float64 underflow (ties)
        L = np.sign(L) * (5.0 + np.abs(L))
    v = (rng.integers(0, 2, N) * (1 - frozen)).astype(np.uint8)
    c = O.encode(v)
    _, x0 = O.sc_decode(L, frozen, fval, fkind)
    _, x1 = O.sc_decode(L * (1.0 - 2.0 * c), frozen, fval, fkind)
    assert np.array_equal(x1, x0 ^ c)


def test_llr_maps():
    y = np.array([0, 1, 1, 0], np.uint8)
    c = math.log(0.98 / 0.02)
    assert O.llr_bsc(y, 0.02).tolist() == [np.float32(c), -np.float32(c), -np.float32(c), np.float32(c)]
    yy = np.array([0.3, -1.7, 2.5])
    assert np.array_equal(O.llr_biawgn(yy, 0.5), (yy * 4.0).astype(np.float32))


# ------------------------------------------------------------------ storage modes
def test_store_fp32_equals_float_decoder():
    rng = np.random.default_rng(123)
    n = 10
    N = 1 << n
    fz = (rng.random(N) < 0.5).astype(np.uint8)
    fv = (rng.integers(0, 2, N) * fz).astype(np.uint8)
    L = rng.normal(0.5, 2.0, N).astype(np.float32)
    for fk in ("minsum", "exact"):
        u0, x0, l0 = O.sc_decode(L, fz, fv, fk, leaf=True)
        u1, x1, l1 = O.sc_decode_store(L, fz, fv, fk, "fp32", leaf=True)
        assert np.array_equal(x0, x1) and np.array_equal(u0, u1) and np.array_equal(l0, l1)


def test_store_rounding_points_n2():
    """N = 2 closed forms of the storage rounding: the g output is stored."""
    _, _, lf = O.sc_decode_store(np.array([1024, 1025], np.float32), [0, 0], [0, 0],
                                 "minsum", "fp16", leaf=True)
    assert lf.tolist() == [1024.0, 2048.0]          # 2049 rounds to even half 2048
    _, _, lf = O.sc_decode_store(np.array([60000, 60000], np.float32), [0, 0], [0, 0],
                                 "minsum", "fp16", leaf=True)
    assert lf.tolist() == [60000.0, 65504.0]        # saturated, not inf
    _, _, lf = O.sc_decode_store(np.array([100, 100], np.float32), [0, 0], [0, 0],
                                 "minsum", "int8", 1.0, leaf=True)
    assert lf.tolist() == [100.0, 127.0]
    _, _, lf = O.sc_decode_store(np.array([2.4, -3.6], np.float32), [0, 0], [0, 0],
                                 "minsum", "int8", 4.0, leaf=True)
    # inputs 9.6 -> 10, -14.4 -> -14; f = -10; u0 = 1 so g = -14 - 10 = -24
    assert lf.tolist() == [-10.0, -24.0]


@pytest.mark.parametrize("store", ["fp16", "int8"])
def test_store_exact_when_nothing_rounds(store):
    """Small-integer LLRs whose partial sums stay within range round nowhere,
    so the reduced-storage decoder equals the float one bit for bit."""
    rng = np.random.default_rng(7)
    n = 6
    N = 1 << n
    for _ in range(50):
        L = rng.integers(-1, 2, N).astype(np.float32)       # |sums| <= 64 < 127
        fz = (rng.random(N) < 0.5).astype(np.uint8)
        fv = (rng.integers(0, 2, N) * fz).astype(np.uint8)
        u0, x0 = O.sc_decode(L, fz, fv, "minsum")
        u1, x1 = O.sc_decode_store(L, fz, fv, "minsum", store, 1.0)
        assert np.array_equal(x0, x1) and np.array_equal(u0, u1)


def test_int8_scale_power_of_two():
    L = np.full(1024, 3.4761, np.float32)
    s = O.int8_scale(L, 8.0)
    assert s == 2.0                  # log2(8 / 3.4761) = 1.20 -> 2^1
    assert O.int8_scale(np.zeros(8, np.float32)) == 1.0
    assert O.int8_scale(np.full(4, 0.01, np.float32), 8.0) == 1024.0
