"""The integer rule the double-float transforms use to split an FP64 value into two floats,
restated on the host and checked against the plain FP64 split (CPU only).

The device split (dd.cuh) reads the bit pattern of v = (-1)^s 2^e (1 + m 2^-52): the high
float keeps the top 23 mantissa bits rounded to nearest even, and the low float is the
remaining 29 bits minus the rounding increment, converted to float and scaled by 2^(e - 52).
That must equal hi = float(v), lo = float(v - hi) for 2^-70 <= |v| < 2^127, keep hi alone
below 2^-70 (an absolute error under 2^-94) and give (0, 0) below FP32's normal range.
The GPU parity tests check the transforms that use it; this test pins the rule itself over
the whole exponent range, ties included."""
import numpy as np


def split_rule(v):
    """Vectorised restatement of the bit-pattern split for |v| < 2^127."""
    b = v.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    sign = ((b >> np.uint64(32)) & np.uint64(0x80000000)).astype(np.uint32)
    mh = ((b >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    rem = (b & np.uint64(0x1FFFFFFF)).astype(np.int64)
    up = ((rem > 0x10000000) | ((rem == 0x10000000) & ((mh & 1) == 1))).astype(np.uint32)
    expf = np.clip(e + 127, 1, 254).astype(np.uint32)
    hi = (sign | ((expf << np.uint32(23)) + mh + up)).view(np.float32)
    diff = rem - np.where(up == 1, 0x20000000, 0)
    scale = np.ldexp(np.float32(1.0), (e - 52).clip(-149, 127)).astype(np.float32)
    lo = (diff.astype(np.float32) * scale).astype(np.float32)  # int -> float rounds to nearest
    lo = np.where(sign != 0, -lo, lo).astype(np.float32)
    tiny = e < -126
    hi = np.where(tiny, np.where(sign != 0, np.float32(-0.0), np.float32(0.0)), hi)
    lo = np.where(tiny | (e < -70), np.float32(0.0), lo)
    return hi.astype(np.float32), lo.astype(np.float32)


def fp64_split(v):
    hi = v.astype(np.float32)
    return hi, (v - hi.astype(np.float64)).astype(np.float32)


def test_split_rule_equals_the_fp64_split():
    rng = np.random.default_rng(7)
    n = 400000
    e = rng.integers(-70, 127, n)
    m = rng.random(n) + 1.0
    v = np.ldexp(m, e) * rng.choice([-1.0, 1.0], n)
    # ties of the high part (remaining 29 bits exactly half) and carries out of the mantissa
    t = rng.integers(0, 1 << 23, 2000).astype(np.uint64)
    ties = ((np.uint64(1023 + 3) << np.uint64(52)) | (t << np.uint64(29)) | np.uint64(0x10000000)).view(np.float64)
    carry = np.ldexp(np.nextafter(2.0, 0.0), rng.integers(-60, 120, 200))
    v = np.concatenate([v, ties, -ties, carry, -carry])
    h1, l1 = split_rule(v)
    h2, l2 = fp64_split(v)
    assert np.array_equal(h1.view(np.uint32), h2.view(np.uint32))
    assert np.array_equal(l1.view(np.uint32), l2.view(np.uint32))


def test_split_rule_below_the_exact_range():
    rng = np.random.default_rng(8)
    v = np.ldexp(rng.random(10000) + 1.0, rng.integers(-126, -70, 10000))
    h, l = split_rule(v)
    assert np.all(l == 0) and np.array_equal(h, v.astype(np.float32))
    err = np.abs(v - h.astype(np.float64))
    assert np.all(err <= 2.0 ** -94)
    h, l = split_rule(np.array([1e-40, -3e-39, 0.0]))
    assert np.all(h == 0) and np.all(l == 0)
