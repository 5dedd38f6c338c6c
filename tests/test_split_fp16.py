"""The arithmetic of the tensor-core deposit's operands, emulated on the host: each FP32 factor
is scaled by a power of two and split into an FP16 head and the FP16 rounding of its exact
rest, and a product is taken as ah bh + ah bt + at bh (the three MMAs).  The column weights
(at most 1) are scaled by 2^14; a row value by 2^s with s chosen from the largest magnitude m
of its accumulation group, m 2^s in [2^14, 2^15) (s at most 100: a group whose largest
magnitude is below 2^-86 keeps less headroom).

Checks: the scaled values never reach the FP16 overflow; the three-product sum reproduces
the FP32 product to about 2^-20 relative wherever the factors are in the FP16 normal range
(the same order as the split-TF32 scheme it replaced); and a factor far below its group's
largest keeps an absolute error below 2^-38 of the largest contribution.
"""
import numpy as np


def group_exp(m):
    """Scale exponent of a group whose largest magnitude is m (m 2^s in [2^14, 2^15))."""
    if not m > 0:
        return 0
    e = int(np.floor(np.log2(np.float32(m))))
    return min(14 - max(e, -126), 100)


def split16(x):
    """FP16 head and FP16 rounding of the exact FP32 rest (both as float64)."""
    x = np.asarray(x, dtype=np.float32)
    h = x.astype(np.float16)
    t = (x - h.astype(np.float32)).astype(np.float16)
    return h.astype(np.float64), t.astype(np.float64)


def split_tf32(x):
    """TF32 head (11 significant bits, rounded) and the TF32 rounding of the rest."""
    x = np.asarray(x, dtype=np.float32)
    bits = x.view(np.uint32)
    h = ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    r = (x - h).astype(np.float32)
    rb = r.view(np.uint32)
    t = ((rb + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    return h.astype(np.float64), t.astype(np.float64)


def split_product(a, b, s):
    """The three-MMA product of row values a (scaled by 2^s) and column weights b (by 2^14),
    unscaled."""
    ah, at = split16(np.float32(2.0 ** s) * np.asarray(a, np.float32))
    bh, bt = split16(np.float32(2.0 ** 14) * np.asarray(b, np.float32))
    return (ah * bh + ah * bt + at * bh) * 2.0 ** (-(s + 14))


def test_scaled_values_stay_below_fp16_overflow():
    rng = np.random.default_rng(1)
    for m in (1e-30, 1e-25, 3.7e-9, 1.0, 12345.0, 3e30):
        a = (rng.uniform(-1, 1, 10000) * m).astype(np.float32)
        a[0] = m
        s = group_exp(np.max(np.abs(a)))
        scaled = np.abs(a.astype(np.float64)) * 2.0 ** s
        if m >= 2.0 ** -86:
            assert 2.0 ** 14 <= scaled.max() < 2.0 ** 15
        else:  # the exponent is capped at 100: smaller groups keep less headroom
            assert s == 100 and 2.0 ** -14 <= scaled.max() < 2.0 ** 15
        h, _ = split16(np.float32(2.0 ** s) * a)
        assert np.all(np.isfinite(h))


def test_three_products_match_fp32_products():
    rng = np.random.default_rng(2)
    n = 200000
    a = (rng.uniform(0.5, 1.0, n) * 10.0 ** rng.uniform(-3, 0, n)).astype(np.float32)
    b = rng.uniform(1e-3, 1.0, n).astype(np.float32)
    s = group_exp(np.max(a))
    exact = a.astype(np.float64) * b.astype(np.float64)
    got = split_product(a, b, s)
    rel = np.abs(got - exact) / exact
    assert rel.max() < 2.0 ** -19
    assert np.sqrt(np.mean(rel ** 2)) < 2.0 ** -21
    # the same order as the split-TF32 scheme the kernel used before
    ah, at = split_tf32(a)
    bh, bt = split_tf32(b)
    rel_tf32 = np.abs(ah * bh + ah * bt + at * bh - exact) / exact
    assert np.sqrt(np.mean(rel ** 2)) < 4 * np.sqrt(np.mean(rel_tf32 ** 2))


def test_faint_factor_error_is_tiny_against_the_group_largest():
    rng = np.random.default_rng(3)
    big = np.float32(1.0)
    faint = (rng.uniform(0.5, 1.0, 1000) * 2.0 ** -30).astype(np.float32)
    b = rng.uniform(0.0, 1.0, 1000).astype(np.float32)
    s = group_exp(big)
    err = np.abs(split_product(faint, b, s) - faint.astype(np.float64) * b.astype(np.float64))
    assert err.max() <= 2.0 ** -38 * float(big)


def test_scale_exponent_plan_is_exact_power_of_two():
    # unscaling by 2^-(s + 14) is exact: a scaled product of FP16 values, in FP64 here, comes
    # back unchanged by the power of two
    for m in (1e-20, 0.3, 1.0, 7e12):
        s = group_exp(m)
        assert -126 <= -(s + 14) <= 127 and -126 <= s <= 127
        x = np.float64(12345.678)
        assert (x * 2.0 ** (-(s + 14))) * 2.0 ** (s + 14) == x
