"""Pins for the oracle's frozen-set construction and capacities (CPU only).

Sec. 3 selects the frozen bits as the least reliable bit-channels found by
density evolution.  The oracle's substitutes (Bhattacharyya recursion for
the BSC, Gaussian approximation for the BI-AWGN channel) are pinned by:
  * the binary erasure channel, where the recursion is exact: brute-force
    enumeration of erasure patterns gives every bit-channel's erasure
    probability, which fixes both the formulas and the index order;
  * conservation sum(1 - Z_i) = N (1 - eps) on the BEC;
  * phi_GA against the numerically integrated true phi, its N = 1 closed
    form P_e = Q(1/sigma), and the defining identity of the minus step;
  * genie-aided Monte Carlo of the (separately pinned) SC decoder;
  * textbook capacities: the BSC threshold p = 0.11 at rate 1/2 and the
    BI-AWGN rate-1/2 Shannon limit Eb/N0 = 0.187 dB.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O


def kron_G(n):
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    for _ in range(n):
        G = np.kron(G, F)
    return G


@pytest.mark.parametrize("eps", [0.2, 0.5, 0.7])
def test_bec_recursion_matches_bruteforce_erasure_probabilities(eps):
    """On the BEC, bit-channel i (genie past) is erased iff some v with
    v_<i = 0, v_i = 1 has v G supported inside the erased positions."""
    n = 3
    N = 1 << n
    G = kron_G(n)
    words = []
    for i in range(N):
        ws = []
        for tail in itertools.product((0, 1), repeat=N - i - 1):
            v = np.zeros(N, np.int64)
            v[i] = 1
            v[i + 1:] = tail
            ws.append(((v @ G) % 2).astype(bool))
        words.append(ws)
    z = np.zeros(N)
    for pattern in itertools.product((0, 1), repeat=N):
        E = np.array(pattern, dtype=bool)
        pr = eps ** E.sum() * (1 - eps) ** (N - E.sum())
        for i in range(N):
            if any(not np.any(c & ~E) for c in words[i]):
                z[i] += pr
    got = np.exp(O.bhatt_log_from(n, math.log(eps)))
    np.testing.assert_allclose(got, z, rtol=1e-12, atol=1e-15)


def test_bec_conservation():
    eps = 0.37
    for n in (4, 10, 14):
        z = np.exp(O.bhatt_log_from(n, math.log(eps)))
        assert (1 - z).sum() == pytest.approx((1 << n) * (1 - eps), rel=1e-9)


def test_bsc_bhattacharyya_z0_and_children():
    p = 0.03
    assert math.exp(O.bhatt_log_bsc(0, p)[0]) == pytest.approx(2 * math.sqrt(p * (1 - p)), rel=1e-14)
    z0 = 2 * math.sqrt(p * (1 - p))
    z1 = np.exp(O.bhatt_log_bsc(1, p))
    assert z1[0] == pytest.approx(2 * z0 - z0 * z0, rel=1e-14)
    assert z1[1] == pytest.approx(z0 * z0, rel=1e-14)
    lz = O.bhatt_log_bsc(12, p)
    assert np.all(lz[1::2] <= lz[0::2])          # Z+ <= Z- for every sibling pair


def test_bsc_bhattacharyya_monotone_in_p():
    a, b = O.bhatt_log_bsc(12, 0.01), O.bhatt_log_bsc(12, 0.05)
    assert np.all(a <= b)


def test_bsc_bhattacharyya_no_underflow_at_2_24():
    lz = O.bhatt_log_bsc(24, 0.02)
    assert np.all(np.isfinite(lz)) and np.all(lz <= 0)
    assert lz.min() < -1e6                        # far below the double range of Z
    assert len(np.unique(lz[-1024:])) > 500


def _phi_true(m):
    """phi(m) = 1 - E[tanh(U/2)], U ~ N(m, 2m) (symmetric Gaussian LLR)."""
    f = lambda u: math.tanh(u / 2) * math.exp(-(u - m) ** 2 / (4 * m)) / math.sqrt(4 * math.pi * m)
    s = 40 * math.sqrt(2 * m)
    v, _ = integrate.quad(f, m - s, m + s, limit=500)
    return 1 - v


@pytest.mark.parametrize("m", [0.2, 0.5, 1.0, 2.0, 5.0, 9.9, 10.1, 20.0, 50.0, 100.0])
def test_ga_phi_close_to_true_phi(m):
    assert math.exp(O.ga_lnphi(m)) == pytest.approx(_phi_true(m), rel=0.06)


def test_ga_phi_is_one_at_zero_and_continuous_at_0867():
    assert O.ga_lnphi(0.0) == 0.0
    assert abs(math.exp(O.ga_lnphi(0.867 - 1e-12)) - math.exp(O.ga_lnphi(0.867))) < 1e-4
    # slope at 0 close to the exact -1/2 (phi(m) = 1 - m/2 + O(m^2))
    assert (math.exp(O.ga_lnphi(1e-4)) - 1.0) / 1e-4 == pytest.approx(-0.5, abs=0.02)


def test_ga_minus_steps_tend_to_zero():
    """Repeated minus steps drive m to 0 (a useless channel), as the true
    density evolution does; a phi with phi(0) > 1 stalls at a positive m."""
    m = O.ga_mean(16, 1.0)
    assert m.min() < 1e-6
    lp = O.ga_lnpe(16, 1.0)
    assert lp[0] > math.log(0.49)            # the all-minus channel is a coin flip


def test_ga_phi_nearly_continuous_at_10():
    assert abs(math.exp(O.ga_lnphi(10.0 - 1e-12)) - math.exp(O.ga_lnphi(10.0))) < 1e-2


@pytest.mark.parametrize("x", [1e-3, 0.5, 3.0, 9.9, 12.0, 100.0, 1e4, 1e7])
def test_ga_lnphi_inverse(x):
    assert O.ga_lnphi_inv(O.ga_lnphi(x)) == pytest.approx(x, rel=1e-11)


@pytest.mark.parametrize("sigma2", [0.3, 1.0, 4.0])
def test_ga_minus_step_identity_and_plus(sigma2):
    m0 = 2.0 / sigma2
    mm, mp = O.ga_mean(1, sigma2)
    assert mp == 2 * m0
    phi0 = math.exp(O.ga_lnphi(m0))
    assert 1 - math.exp(O.ga_lnphi(mm)) == pytest.approx((1 - phi0) ** 2, rel=1e-10)


@pytest.mark.parametrize("sigma2", [0.25, 1.0, 2.0])
def test_ga_single_channel_is_exact_biawgn_error(sigma2):
    want = math.log(0.5 * math.erfc(1 / math.sqrt(2 * sigma2)))
    assert O.ga_lnpe(0, sigma2)[0] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("x", [0.0, 1.0, 5.0, 29.9, 30.1, 100.0, 1000.0])
def test_ln_q(x):
    assert O.ln_q(x) == pytest.approx(special.log_ndtr(-x), rel=1e-9)


def test_ga_no_underflow_at_2_24_subset():
    lp = O.ga_lnpe(16, 1.0)
    assert np.all(np.isfinite(lp)) and np.all(lp < 0)


def _genie_error_rates(n, channel, param, T, seed):
    """Bit-channel error rates of SC with a genie (every position frozen to
    the true u), counted from the leaf LLR signs; L = 0 counts one half."""
    N = 1 << n
    rng = np.random.default_rng(seed)
    err = np.zeros(N)
    allf = np.ones(N, np.uint8)
    for _ in range(T):
        x = rng.integers(0, 2, N).astype(np.uint8)
        if channel == "bsc":
            L = O.llr_bsc(x ^ (rng.random(N) < param).astype(np.uint8), param, 64)
        else:
            L = O.llr_biawgn((1.0 - 2.0 * x) + math.sqrt(param) * rng.standard_normal(N), param, 64)
        u = O.encode(x)
        _, _, leaf = O.sc_decode(L, allf, u, "exact", leaf=True)
        err += np.where(leaf == 0, 0.5, ((leaf < 0) != (u == 1)) * 1.0)
    return err / T


def test_ga_matches_genie_monte_carlo():
    n, s2, T = 8, 1.0, 3000
    pe = _genie_error_rates(n, "biawgn", s2, T, 11)
    ga = np.exp(O.ga_lnpe(n, s2))
    sel = (ga > 0.01) & (ga < 0.3)
    assert sel.sum() > 40
    ratio = pe[sel] / ga[sel]
    assert np.all(ratio > 0.5) and np.all(ratio < 2.0)


def test_bhattacharyya_bounds_genie_monte_carlo():
    n, p, T = 8, 0.05, 3000
    pe = _genie_error_rates(n, "bsc", p, T, 12)
    z = np.exp(O.bhatt_log_bsc(n, p))
    se = np.sqrt(np.maximum(pe * (1 - pe), 1.0 / T) / T)
    assert np.all(pe <= z + 3 * se)
    # the bound orders channels usefully: the better half has lower error
    order = np.argsort(z)
    assert pe[order[: 1 << (n - 1)]].mean() < pe[order[1 << (n - 1):]].mean()


def test_select_frozen_rule():
    bad = np.array([0.0, -1.0, 5.0, 5.0, -3.0, 5.0, 2.0, -1.0])
    fz = O.select_frozen(bad, 4)
    # freeze the 4 largest; ties among the 5.0's and the rule "lower index first"
    assert fz.tolist() == [0, 0, 1, 1, 0, 1, 1, 0]
    fz = O.select_frozen(np.zeros(8), 5)
    assert fz.tolist() == [1, 1, 1, 0, 0, 0, 0, 0]
    assert O.select_frozen(bad, 8).sum() == 0 and O.select_frozen(bad, 0).sum() == 8


def test_frozen_set_counts():
    fz, K = O.frozen_set(16, "bsc", 0.02, 0.80)
    assert K == 52428 and int((fz == 0).sum()) == K
    fz, K = O.frozen_set(12, "biawgn", 1.0, 0.44)
    assert K == int(0.44 * 4096) and int((fz == 0).sum()) == K


def test_capacity_textbook_values():
    assert O.capacity("bsc", 0.11) == pytest.approx(0.5, abs=1e-3)
    assert O.capacity("bsc", 0.5) == pytest.approx(0.0, abs=1e-12)
    ebn0 = 10 ** (0.187 / 10)                # rate-1/2 BI-AWGN Shannon limit
    sigma2 = 1.0 / (2 * 0.5 * ebn0)
    assert O.capacity("biawgn", sigma2) == pytest.approx(0.5, abs=1e-3)
    assert O.capacity("biawgn", 1e-3) == pytest.approx(1.0, abs=1e-9)
    assert O.capacity("biawgn", 1.0) < O.capacity("biawgn", 0.9)
