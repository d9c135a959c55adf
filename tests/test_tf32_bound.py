"""The rounding bounds behind the tensor-core contraction tests, on a numpy
emulation of float32 -> TF32 round-to-nearest (ties away from zero: keep the
sign, the exponent and the 10 leading mantissa bits, rounding on the 13
dropped ones).

* one operand: |tf32(x) - x| <= 2^-11 |x|;
* one product term of two rounded operands: |tf32(a) tf32(b) - a b| <= (2^-10 + 2^-22) |a b|;
* a dot product of such terms: the error is at most (2^-10 + 2^-22) sum |a_i b_i| (relative
  to |sum a_i b_i| where the terms share a sign, as the density's products with the
  nonnegative kernels and likelihoods do);
* the split operand hi = tf32(x), lo = tf32(x - hi): |hi + lo - x| <= 2^-22 |x|, and the three
  split products hi*hi + hi*lo + lo*hi miss a b by at most 2^-20 |a b|.
"""
import numpy as np

U11 = 2.0 ** -11


def tf32(x):
    """Round float32 values to TF32 (10 explicit mantissa bits), to nearest,
    ties away from zero; the result is a float32 with the 13 low bits zero."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    sign = b & 0x80000000
    mag = b & 0x7FFFFFFF
    mag = (mag + 0x1000) & ~np.uint64(0x1FFF)
    return (sign | mag).astype(np.uint32).view(np.float32)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    # magnitudes across the normal float32 range, both signs
    return (rng.standard_normal(n) * np.exp2(rng.integers(-100, 100, n))).astype(np.float32)


def test_emulation_keeps_ten_mantissa_bits():
    x = _samples(100000, 1)
    t = tf32(x)
    assert (t.view(np.uint32) & 0x1FFF == 0).all()
    # values already in TF32 are kept; a tie rounds away from zero
    assert (tf32(t) == t).all()
    one_and_half_ulp = np.float32(1.0 + 2.0 ** -11)  # halfway between 1 and 1 + 2^-10
    assert tf32(one_and_half_ulp) == np.float32(1.0 + 2.0 ** -10)
    assert tf32(-one_and_half_ulp) == -np.float32(1.0 + 2.0 ** -10)


def test_operand_and_product_bounds():
    a, b = _samples(200000, 2), _samples(200000, 3)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    ta, tb = tf32(a).astype(np.float64), tf32(b).astype(np.float64)
    assert (np.abs(ta - a64) <= U11 * np.abs(a64)).all()
    rel = np.abs(ta * tb - a64 * b64) / np.abs(a64 * b64)
    assert (rel <= 2.0 ** -10 + 2.0 ** -22).all()
    assert rel.max() > 0.9 * 2.0 ** -10  # and it is nearly reached: not a loose bound


def test_dot_product_bound():
    rng = np.random.default_rng(4)
    for k in (16, 144, 1024):
        a = rng.standard_normal((200, k)).astype(np.float32)
        b = rng.standard_normal((200, k)).astype(np.float32)
        exact = (a.astype(np.float64) * b.astype(np.float64)).sum(1)
        got = (tf32(a).astype(np.float64) * tf32(b).astype(np.float64)).sum(1)
        mag = np.abs(a.astype(np.float64) * b.astype(np.float64)).sum(1)
        assert (np.abs(got - exact) <= (2.0 ** -10 + 2.0 ** -22) * mag).all()
        # nonnegative terms: the bound relative to the result itself
        pa, pb = np.abs(a), np.abs(b)
        ex = (pa.astype(np.float64) * pb).sum(1)
        gt = (tf32(pa).astype(np.float64) * tf32(pb).astype(np.float64)).sum(1)
        assert (np.abs(gt - ex) <= (2.0 ** -10 + 2.0 ** -22) * ex).all()


def test_split_operands_reach_float32_level():
    a, b = _samples(200000, 5), _samples(200000, 6)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    ah = tf32(a)
    al = tf32((a - ah).astype(np.float32))  # x - hi is exact in float32
    assert ((a - ah).astype(np.float64) == a64 - ah.astype(np.float64)).all()
    assert (np.abs(ah.astype(np.float64) + al - a64) <= 2.0 ** -22 * np.abs(a64)).all()
    bh = tf32(b)
    bl = tf32((b - bh).astype(np.float32))
    ah, al, bh, bl = (v.astype(np.float64) for v in (ah, al, bh, bl))
    three = ah * bh + ah * bl + al * bh
    assert (np.abs(three - a64 * b64) <= 2.0 ** -20 * np.abs(a64 * b64)).all()
