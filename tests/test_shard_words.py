"""CPU pins of the exchange-word codec the sharded tests use (tests/shard_words.py): the decoded
total of values whose truncation to 2^-96 is exact is their correctly rounded sum (math.fsum),
splitting the values over several shards' words changes nothing, two's complement carries
through negative totals, and non-finite or huge values are counted, not added."""
import math
import random

import numpy as np

import shard_words


def _values(rng, n):
    # |v| >= 2^-40 with 53-bit significands: every ulp is >= 2^-92, so truncation is exact
    return [rng.choice([-1.0, 1.0]) * math.ldexp(rng.random() + 0.5, rng.randint(-40, 60)) for _ in range(n)]


def test_decoded_total_is_the_correctly_rounded_sum():
    rng = random.Random(11)
    for n in (1, 7, 1000):
        v = _values(rng, n)
        D, E, f, members, shards = shard_words.decode(shard_words.encode(v))
        assert D == math.fsum(v)
        assert E == 0.0 and f == (0, 0, 0, 0) and members == n and shards == 1


def test_split_words_add_to_the_whole():
    rng = random.Random(12)
    v = _values(rng, 999)
    whole = shard_words.decode(shard_words.encode(v))
    for cuts in ([0, 999], [0, 1, 999], [0, 333, 334, 998, 999], [0, 100, 200, 300, 999]):
        parts = [shard_words.encode(v[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
        total = np.sum(np.stack(parts), axis=0)
        D, E, f, members, shards = shard_words.decode(total)
        assert (D, E, f, members) == whole[:4]
        assert shards == len(parts)


def test_negative_totals_and_truncation_toward_zero():
    D = shard_words.decode(shard_words.encode([-1.5, -2.25, 0.125]))[0]
    assert D == -3.625
    tiny = math.ldexp(1.0, -97)  # below the resolution: contributes nothing, either sign
    assert shard_words.decode(shard_words.encode([tiny, -tiny, 1.0]))[0] == 1.0
    v = -math.ldexp(1.0 + 2.0 ** -52, -96)  # truncates toward zero to -2^-96
    assert shard_words.decode(shard_words.encode([v]))[0] == -math.ldexp(1.0, -96)
    # a total of -2^-96 exactly: all 192 bits set
    w = shard_words.encode([-math.ldexp(1.0, -96)])
    assert all(int(q) == 0xFFFFFFFF for q in w[:6])


def test_non_finite_and_huge_values_are_counted():
    v = [1.0, -math.inf, math.nan, 2.0 ** 95, -(2.0 ** 94), 3.0]
    D, E, f, members, _ = shard_words.decode(shard_words.encode(v, e_terms=[0.5, math.nan]))
    assert D == 4.0 and E == 0.5
    assert f == (2, 2, 1, 0)  # f0: -inf and -2^94; f1: the d NaN and the selection term's NaN
    assert members == 6
