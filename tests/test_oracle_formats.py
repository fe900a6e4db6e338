"""Pins of the oracle's update storage formats (reduced-precision bins).

Expected bit patterns are written out from the IEEE 754 binary16 layout
(1 sign, 5 exponent bits with bias 15, 10 fraction bits) and the bfloat16
layout (binary32's upper half: 1 sign, 8 exponent bits with bias 127, 7
fraction bits), with round to nearest, ties to even."""
import numpy as np

import oracle

S = 2.0 ** -15  # the FP16 format stores value * 2^15


def f16_bits(values):
    return oracle.store_updates(np.asarray(values, np.float32), "f16").view(np.uint16).tolist()


def bf16_bits(values):
    return oracle.store_updates(np.asarray(values, np.float32), "bf16").tolist()


def test_f16_exact_values():
    # 1.0 = 0x3C00, 2.0 = 0x4000, 0.5 = 0x3800, 1.5 = 0x3E00, 0 = 0x0000
    assert f16_bits([1 * S, 2 * S, 0.5 * S, 1.5 * S, 0.0]) == [0x3C00, 0x4000, 0x3800, 0x3E00, 0x0000]


def test_f16_rounds_to_nearest_even():
    ulp = 2.0 ** -10  # spacing of binary16 in [1, 2)
    # exactly halfway between 1 and 1 + ulp: ties to the even fraction (1.0)
    # just above halfway rounds up; halfway between 1 + ulp and 1 + 2 ulp goes to 1 + 2 ulp
    vals = [(1 + ulp / 2) * S, (1 + ulp / 2 + 2.0 ** -20) * S, (1 + 1.5 * ulp) * S]
    assert f16_bits(vals) == [0x3C00, 0x3C01, 0x3C02]


def test_f16_saturates_and_keeps_subnormals():
    # SPR = 4 would scale to 2^17 > 65504: stored as 65504 = 0x7BFF, not infinity
    assert f16_bits([4.0, 65504 * S]) == [0x7BFF, 0x7BFF]
    # the smallest binary16 subnormal is 2^-24: stored value 2^-24 -> 0x0001
    assert f16_bits([2.0 ** -24 * S]) == [0x0001]
    # changes of SPR (delta iterations) are signed: -65504 = 0xFBFF saturates
    # the other way, -1.0 = 0xBC00, -2^-24 = 0x8001
    assert f16_bits([-4.0, -1 * S, -(2.0 ** -24) * S]) == [0xFBFF, 0xBC00, 0x8001]


def test_bf16_exact_and_ties():
    ulp = 2.0 ** -7  # spacing of bfloat16 in [1, 2)
    vals = [1.0, -2.0, 1 + ulp / 2, 1 + 1.5 * ulp, 1 + ulp / 2 + 2.0 ** -20, 0.0]
    # 1.0 = 0x3F80, -2.0 = 0xC000, ties to even: 0x3F80 and 0x3F82, above the tie: 0x3F81
    assert bf16_bits(vals) == [0x3F80, 0xC000, 0x3F80, 0x3F82, 0x3F81, 0x0000]


def test_load_inverts_store_within_half_an_ulp():
    rng = np.random.default_rng(3)
    v = (rng.random(10000) * 1e-3).astype(np.float32)
    for dtype, rel in (("f16", 2.0 ** -11), ("bf16", 2.0 ** -8), ("f32", 0.0)):
        back = oracle.load_updates(oracle.store_updates(v, dtype), dtype)
        err = np.abs(back - v.astype(np.float64))
        assert np.all(err <= rel * np.abs(v.astype(np.float64)) + (2.0 ** -24 * S if dtype == "f16" else 0.0)), dtype
