"""Exchange words of one shard's sweep, encoded and decoded on the CPU from their definition in
the C header (CUDAHM_SHARD_WORDS): words 0-5 hold D = sum_i d_i and words 6-11 the selection
integral, each as the six 32-bit limbs (low first) of a 192-bit two's-complement fixed-point
number with 2^-96 resolution, every addend truncated toward zero to a multiple of 2^-96; word 12
is the count of d_i <= -2^94 (or -inf) plus the NaN count times 2^32; word 13 the count of
d_i >= 2^94 plus the member-step NaN count times 2^32; word 14 the shard's member count; word 15
is 1. The words of several shards add as integers (an all-reduce with the sum operation).

Python integers stand in for the fixed-point arithmetic: math.ldexp scales a binary64 value by
2^96 exactly and int() truncates toward zero, and int / int is correctly rounded, as the
device's round-to-nearest-even conversion of the total is.
"""
import math

import numpy as np

WORDS = 16
BIG = 2.0 ** 94
_MASK = (1 << 192) - 1


def _fixed_sum(values, flags):
    """Exact sum of the truncated fixed-point addends; non-finite or huge values are counted."""
    x = 0
    for v in values:
        v = float(v)
        if math.isnan(v):
            flags["nan"] += 1
        elif v <= -BIG:
            flags["neg"] += 1
        elif v >= BIG:
            flags["pos"] += 1
        else:
            x += int(math.ldexp(v, 96))
    return x


def encode(d, e_terms=(), n_members=None) -> np.ndarray:
    """The words of one shard: its d_i, its terms of the selection integral, its member count."""
    flags = {"nan": 0, "neg": 0, "pos": 0}
    x = _fixed_sum(d, flags) & _MASK
    ef = {"nan": 0, "neg": 0, "pos": 0}
    e = _fixed_sum(e_terms, ef) & _MASK
    w = [0] * WORDS
    for k in range(6):
        w[k] = (x >> (32 * k)) & 0xFFFFFFFF
        w[6 + k] = (e >> (32 * k)) & 0xFFFFFFFF
    nan = flags["nan"] + ef["nan"] + ef["neg"] + ef["pos"]
    w[12] = flags["neg"] | (nan << 32)
    w[13] = flags["pos"]
    w[14] = len(d) if n_members is None else int(n_members)
    w[15] = 1
    return np.array(w, dtype=np.int64)


def _value(words, k0):
    v = 0
    for k in range(6):
        v += int(words[k0 + k]) << (32 * k)  # limb sums carry into the next limb here
    v &= _MASK
    if v >> 191:
        v -= 1 << 192
    return v


def decode(words):
    """(D, E, (f0, f1, f2, f3), members, shards) of summed words; D and E correctly rounded."""
    w = [int(q) & 0xFFFFFFFFFFFFFFFF for q in np.asarray(words).tolist()]
    D = _value(w, 0) / (1 << 96)
    E = _value(w, 6) / (1 << 96)
    f = (w[12] & 0xFFFFFFFF, w[12] >> 32, w[13] & 0xFFFFFFFF, w[13] >> 32)
    return D, E, f, w[14], w[15]
