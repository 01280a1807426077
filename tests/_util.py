"""Test helpers: conversions between the oracle's per-value flags and the library's bitsets.

These are test infrastructure; they hold no propagation or search arithmetic.
"""
import numpy as np


def flags_to_bits(om, flags, n, W, lo0):
    """Oracle flags (value lo_i + k of var i) -> n*W uint32 words (bit b = value lo0 + b)."""
    words = np.zeros(n * W, dtype=np.uint32)
    for i in range(n):
        for k in range(int(om.size[i])):
            if flags[om.off[i] + k]:
                b = int(om.lo[i]) + k - lo0
                words[i * W + b // 32] |= np.uint32(1 << (b % 32))
    return words


def bits_to_flags(om, words, n, W, lo0):
    f = np.zeros(int(om.off[-1]), dtype=np.uint8)
    for i in range(n):
        for k in range(int(om.size[i])):
            b = int(om.lo[i]) + k - lo0
            if (int(words[i * W + b // 32]) >> (b % 32)) & 1:
                f[om.off[i] + k] = 1
    return f


def random_subdomains(om, rng, count, p_lo=0.4, p_hi=0.95):
    base = om.root_flags()
    out = []
    for _ in range(count):
        p = rng.uniform(p_lo, p_hi)
        keep = rng.random(base.shape[0]) < p
        f = (base & keep).astype(np.uint8)
        out.append(f)
    return out


def sorted_rows(a):
    return sorted(map(tuple, np.asarray(a).tolist()))
