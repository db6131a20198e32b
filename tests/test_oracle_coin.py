"""Pins of the oracle's Philox4x64-10 coin against numpy's independent implementation."""

import numpy as np
import pytest

from oracle import coin

MASK = (1 << 64) - 1


def _numpy_block(counter, key):
    """numpy's Philox bit generator increments its counter before producing a block,
    so the block for counter c comes from a generator started at c - 1 (mod 2^256)."""
    c = list(counter)
    i = 0
    while True:  # subtract one with borrow across the four words
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = MASK
        i += 1
        if i == 4:
            break
    g = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return [int(x) for x in g.random_raw(4)]


@pytest.mark.parametrize("seed", [0, 1, 7, 12345, 2**63 + 5, MASK])
def test_philox_matches_numpy(seed):
    for k in list(range(0, 40)) + [1000, 2**32 - 1, 2**32, 2**40 + 3]:
        assert coin.philox4x64_10((k, 0, 0, 0), (seed, 0)) == _numpy_block((k, 0, 0, 0), (seed, 0))


def test_philox_matches_numpy_general_words():
    ctr = (0x0123456789ABCDEF, 0xFEDCBA9876543210, 0x1111, 0xFFFFFFFFFFFFFFFF)
    key = (0xDEADBEEFCAFEF00D, 0x0F0F0F0F0F0F0F0F)
    assert coin.philox4x64_10(ctr, key) == _numpy_block(ctr, key)


@pytest.mark.parametrize("p", [0.05, 0.1, 0.3, 0.5, 0.9])
def test_coin_binomial_mean(p):
    """Sum of K coins is Binomial(K, p): within 5 standard deviations."""
    K = 20000
    s = sum(coin.schedule(3, p, K))
    assert abs(s - K * p) <= 5.0 * np.sqrt(K * p * (1 - p))


def test_coin_degenerate_and_invalid():
    assert all(coin.schedule(11, 1.0, 2000))
    for bad in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(ValueError):
            coin.coin(0, bad, 0)


def test_coin_threshold_is_exact():
    """theta = [(w >> 11) < p 2^53]: check the boundary on a hand-picked word."""
    w = coin.philox4x64_10((5, 0, 0, 0), (9, 0))[0]
    u53 = w >> 11
    p_hit = (u53 + 1) / 2.0 ** 53      # u53 < p 2^53 holds
    p_miss = u53 / 2.0 ** 53           # u53 < p 2^53 fails
    assert coin.coin(9, p_hit, 5) == 1
    if p_miss > 0:
        assert coin.coin(9, p_miss, 5) == 0
