"""Pins for the oracle's degraded-channel (Tal-Vardy) construction and the
Sec. 3 rate rule (CPU only).

The construction makes Sec. 3's density evolution finite: each bit-channel
is tracked as a channel with at most mu outputs, merged so that it is always
degraded with respect to the true bit-channel.  Pinned by:
  * brute-force bit-channel ML error probabilities of the BSC at N <= 8,
    which the construction must reproduce exactly when mu is large enough
    that nothing is merged (this fixes the minus / plus formulas and the
    index order), and bound from above when merging is forced;
  * the BI-AWGN starting quantisation, whose sign decision is exact:
    its error probability is Q(1/sigma) whatever the bins;
  * genie-aided Monte Carlo of the (separately pinned) SC decoder;
  * the rate rule: K is the largest count whose most reliable channels sum
    to at most the target, checked by brute force on small arrays.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special

import oracle as O


def kron_G(n):
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    for _ in range(n):
        G = np.kron(G, F)
    return G


def bruteforce_pe_bsc(n, p):
    """ML error probability of every bit-channel W_i(y, u_<i | u_i) of the
    BSC(p) with uniform u, by enumeration of all u and y."""
    N = 1 << n
    G = kron_G(n)
    us = np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.int64)   # u_0 first
    xs = (us @ G) % 2
    ys = us.copy()                                                            # all outputs
    d = (xs[:, None, :] != ys[None, :, :]).sum(-1)                            # [u, y]
    W = p ** d * (1 - p) ** (N - d)
    pe = np.zeros(N)
    for i in range(N):
        # index of u = sum u_j 2^(N-1-j): u_<i are the top i bits
        Wi = W.reshape(2 ** i, 2, 2 ** (N - i - 1), 2 ** N).sum(axis=2) / 2 ** (N - 1)
        pe[i] = 0.5 * np.minimum(Wi[:, 0, :], Wi[:, 1, :]).sum()
    return pe


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("p", [0.02, 0.11, 0.3])
def test_tv_exact_when_nothing_is_merged(n, p):
    got = O.tv_pe(n, "bsc", p, mu=128)
    np.testing.assert_allclose(got, bruteforce_pe_bsc(n, p), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("p", [0.05, 0.2])
def test_tv_merging_bounds_from_above(p):
    exact = bruteforce_pe_bsc(3, p)
    for mu in (2, 4, 8):
        got = O.tv_pe(3, "bsc", p, mu=mu)
        assert np.all(got >= exact - 1e-15), mu
    assert np.any(O.tv_pe(3, "bsc", p, mu=2) > exact + 1e-6)   # merging did happen


@pytest.mark.parametrize("sigma2", [0.25, 1.0, 4.0])
@pytest.mark.parametrize("mu", [2, 16, 64])
def test_tv_biawgn_start_keeps_the_sign_decision(sigma2, mu):
    q = 0.5 * special.erfc(1.0 / math.sqrt(2 * sigma2))
    assert O.tv_pe(0, "biawgn", sigma2, mu=mu)[0] == pytest.approx(q, rel=1e-12)


def test_tv_polarises_and_conserves_extremes():
    pe = O.tv_pe(12, "bsc", 0.03, 16)
    assert pe[0] == pytest.approx(0.5, abs=1e-9)       # minus^12: useless
    assert pe[-1] < 1e-100                              # plus^12: perfect
    assert np.all((pe >= 0) & (pe <= 0.5 + 1e-12))


def test_tv_bounds_and_tracks_genie_monte_carlo():
    """Upper bound on the genie error rates (within Monte Carlo error), and
    tight: channels with rates in [0.01, 0.3] agree within a factor 1.5."""
    from test_oracle_construction import _genie_error_rates
    n, p, T = 8, 0.05, 3000
    mc = _genie_error_rates(n, "bsc", p, T, 12)
    tv = O.tv_pe(n, "bsc", p, 32)
    se = np.sqrt(np.maximum(mc * (1 - mc), 1.0 / T) / T)
    assert np.all(mc <= tv + 3 * se)
    sel = (tv > 0.01) & (tv < 0.3)
    assert sel.sum() > 30
    r = mc[sel] / tv[sel]
    assert np.all(r > 1 / 1.5) and np.all(r < 1.5)


def test_tv_ranks_bsc_channels_better_than_the_bhattacharyya_bound():
    """At a rate above the Bhattacharyya bound's reach (R = 0.75 at p = 0.03,
    whose bound behaves like a BEC of capacity 0.66), the degraded set's
    information bits have a far smaller genie error sum."""
    from test_oracle_construction import _genie_error_rates
    n, p, T = 10, 0.03, 300
    mc = _genie_error_rates(n, "bsc", p, T, 21)
    K = int(0.75 * (1 << n))
    fz_tv = O.select_frozen(O.tv_pe(n, "bsc", p, 16), K)
    fz_bh = O.select_frozen(O.bhatt_log_bsc(n, p), K)
    assert mc[fz_tv == 0].sum() < 0.5 * mc[fz_bh == 0].sum()


def test_k_for_sum_rule_bruteforce():
    rng = np.random.default_rng(4)
    for _ in range(20):
        bad = rng.exponential(0.01, 16)
        bad[rng.integers(0, 16, 3)] = 0.02                 # ties
        for target in (0.0, 0.005, 0.03, 0.1, 10.0):
            K = O.k_for_sum(bad, target)
            # the information set of size K is the complement of select_frozen's
            fz = O.select_frozen(bad, K)
            assert bad[fz == 0].sum() <= target + 1e-15
            if K < 16:
                fz2 = O.select_frozen(bad, K + 1)
                assert bad[fz2 == 0].sum() > target


def test_k_for_sum_log_rule_bruteforce():
    rng = np.random.default_rng(5)
    for _ in range(20):
        lb = np.log(rng.exponential(0.01, 16))
        lb[rng.integers(0, 16, 3)] = math.log(0.02)
        for target in (0.0, 0.005, 0.03, 0.1, 10.0):
            K = O.k_for_sum_log(lb, target)
            fz = O.select_frozen(lb, K)
            assert np.exp(lb[fz == 0]).sum() <= target * (1 + 1e-12)
            if K < 16:
                assert np.exp(lb[O.select_frozen(lb, K + 1) == 0]).sum() > target


def test_frozen_set_sum_mode():
    fz, K, s = O.frozen_set_sum(12, "biawgn", 1.0, 0.1)
    assert int((fz == 0).sum()) == K and s <= 0.1
    assert O.frozen_set_sum(12, "biawgn", 1.0, 1.0)[1] > K


def test_frozen_set_tv_modes():
    fz, K, s = O.frozen_set_tv(12, "biawgn", 1.0, sum_pe_max=0.1)
    assert int((fz == 0).sum()) == K and s <= 0.1
    fz2, K2, s2 = O.frozen_set_tv(12, "biawgn", 1.0, rate=0.44)
    assert K2 == int(0.44 * 4096) and int((fz2 == 0).sum()) == K2
