"""The integer-pipe maxima of the kernels, checked on the CPU.

Column norms and scaled offsets are non-negative doubles.  csrc/la.cuh reduces them as 64-bit keys (their
bit patterns), so that the team maxima run on the integer pipe instead of the FP64 pipe, which costs
about 80 cycles per warp instruction on this GPU.  The warp reduction splits a key into 32-bit halves:
the high halves are reduced first, then the low halves of only the lanes that hold that high half, and
for the arg-max the smallest index among the lanes that hold both.  The team stage then compares the
warps' partial keys, ties going to the smaller index.  Restated here and compared with the plain
definition (the largest value, its smallest index) on random and adversarial inputs.
"""
import struct

import numpy as np


def key(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def value(k):
    return struct.unpack("<d", struct.pack("<Q", k))[0]


def warp_argmax(keys, idx):
    """la.cuh warp_argmax_key over 32 lanes: (key, index) of the warp's best."""
    hi = [k >> 32 for k in keys]
    lo = [k & 0xFFFFFFFF for k in keys]
    mhi = max(hi)
    mlo = max(l if h == mhi else 0 for h, l in zip(hi, lo))
    widx = min(i if (h == mhi and l == mlo) else 0x7FFFFFFF for h, l, i in zip(hi, lo, idx))
    return (mhi << 32) | mlo, widx


def team_argmax(vals, idx, warps):
    """warp stage on each warp's 32 lanes, then la.cuh argmax_finish over the warps."""
    parts = [warp_argmax([key(v) for v in vals[32 * w:32 * w + 32]], idx[32 * w:32 * w + 32]) for w in range(warps)]
    best, besti = parts[0]
    for k2, i2 in parts[1:]:
        if k2 > best or (k2 == best and i2 < besti):
            best, besti = k2, i2
    return value(best), besti


def test_key_order_is_value_order_for_non_negative_doubles():
    rng = np.random.default_rng(0)
    special = [0.0, 5e-324, 2.2250738585072014e-308, 1e-300, 1.0, 1.0000000000000002, 1e300, float("inf")]
    vals = special + list(np.abs(rng.standard_normal(2000)) * 10.0 ** rng.integers(-300, 300, 2000))
    vals = [float(v) for v in vals]
    order_v = sorted(range(len(vals)), key=lambda i: (vals[i], i))
    order_k = sorted(range(len(vals)), key=lambda i: (key(vals[i]), i))
    assert order_v == order_k


def test_two_stage_arg_max_is_the_largest_value_with_the_smallest_index():
    rng = np.random.default_rng(1)
    for trial in range(3000):
        warps = int(rng.choice([1, 2, 4, 8]))
        n = 32 * warps
        kind = trial % 4
        if kind == 0:    # random magnitudes
            vals = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-20, 20, n)
        elif kind == 1:  # many exact ties
            vals = rng.integers(0, 4, n).astype(float)
        elif kind == 2:  # equal high halves, different low halves
            base = key(1.5)
            vals = np.array([value(base + int(d)) for d in rng.integers(0, 1 << 20, n)])
        else:            # lanes that do not hold a candidate carry key 0
            vals = np.where(rng.random(n) < 0.7, 0.0, np.abs(rng.standard_normal(n)))
        vals = [float(v) for v in vals]
        idx = [int(i) for i in rng.permutation(n)]  # column indices need not follow the lanes
        bv, bi = team_argmax(vals, idx, warps)
        top = max(vals)
        assert bv == top
        assert bi == min(i for v, i in zip(vals, idx) if v == top)
