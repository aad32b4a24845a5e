"""Detailed balance of the oracle's member accept rule on a two-state target (no GPU needed).

Sec. 2.2's member step accepts with probability min(1, pi(Y)/pi(X)). On the states {0, 1} with
target (pi0, pi1) = (1 - pi1, pi1) and a proposal that always flips (symmetric), the chain has
P01 = min(1, pi1/pi0), P10 = min(1, pi0/pi1), detailed balance pi0 P01 = pi1 P10 and the
stationary occupation pi1 of state 1. The oracle's two-state chains use the member step's
accept (ln u < Delta) and its accept uniform; each estimated quantity must lie within 5 sigma of
its exact value, and an exact 1 (an uphill or level move) must hold in every step. A flipped
sign of Delta, a reversed comparison or a uniform from the wrong range fails these.
"""
import math

import numpy as np
import pytest

import oracle


def check_detailed_balance(c, pi1, sweeps, z=5.0):
    """c = [[n00, n01], [n10, n11]] transition counts of flip-proposal chains on (1 - pi1, pi1),
    each run for `sweeps` steps from state 0 or 1."""
    pi0 = 1.0 - pi1
    n0, n1 = c[0].sum(), c[1].sum()
    assert n0 > 0 and n1 > 0
    p01, p10 = min(1.0, pi1 / pi0), min(1.0, pi0 / pi1)
    h01, h10 = c[0, 1] / n0, c[1, 0] / n1
    s01 = math.sqrt(p01 * (1 - p01) / n0)
    s10 = math.sqrt(p10 * (1 - p10) / n1)
    if p01 == 1.0:
        assert c[0, 0] == 0, "an uphill or level move was rejected"
    else:
        assert abs(h01 - p01) <= z * s01, (h01, p01, s01)
    if p10 == 1.0:
        assert c[1, 1] == 0, "an uphill or level move was rejected"
    else:
        assert abs(h10 - p10) <= z * s10, (h10, p10, s10)
    # detailed balance with the estimated probabilities
    sdb = math.sqrt((pi0 * s01) ** 2 + (pi1 * s10) ** 2)
    assert abs(pi0 * h01 - pi1 * h10) <= z * sdb + 1e-15
    # stationary occupation of state 1: the asymptotic variance of a two-state chain's mean, plus
    # the start's pull (a chain started off stationarity deviates by at most sum |lam|^k / sweeps)
    lam = 1.0 - p01 - p10
    steps = n0 + n1
    socc = math.sqrt(pi0 * pi1 * (1 + lam) / max(1e-12, 1 - lam) / steps)
    start = (1.0 if abs(lam) == 1.0 else 1.0 / (1.0 - abs(lam))) / sweeps  # |lam| = 1: the chain alternates
    assert abs(n1 / steps - pi1) <= z * socc + start, (n1 / steps, pi1, socc, start)


@pytest.mark.parametrize("pi1", [0.7, 0.2, 0.5, 0.999])
def test_oracle_two_state_chains_satisfy_detailed_balance(pi1):
    c = oracle.twostate_counts(pi1, 2000, 1000, seed=5)
    assert c.sum() == 2000 * 1000
    check_detailed_balance(c, pi1, 1000)


def test_level_target_accepts_every_flip():
    c = oracle.twostate_counts(0.5, 100, 200, seed=6)
    assert c[0, 0] == 0 and c[1, 1] == 0 and c.sum() == 20000


def test_check_rejects_a_wrong_rule():
    """The check itself: counts from a sampler with the comparison reversed (accept iff
    ln u > Delta) fail it."""
    rng = np.random.default_rng(7)
    pi1, c = 0.7, np.zeros((2, 2), dtype=np.int64)
    lp = np.log([0.3, 0.7])
    x = np.arange(4000) & 1
    for _ in range(200):
        u = rng.random(x.size)
        acc = np.log(u) > lp[1 - x] - lp[x]
        y = np.where(acc, 1 - x, x)
        np.add.at(c, (x, y), 1)
        x = y
    with pytest.raises(AssertionError):
        check_detailed_balance(c, pi1, 200)
