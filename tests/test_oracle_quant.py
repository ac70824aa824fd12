"""Pins of the BF16 / E4M3 restatements against the formats' definitions."""

import numpy as np

from oracle import quant


def test_bf16_known_patterns_and_ties():
    assert quant.bf16_encode(1.0) == 0x3F80
    assert quant.bf16_encode(-2.0) == 0xC000
    assert quant.bf16_encode(1.0 + 2 ** -8) == 0x3F80           # halfway: to even (0x3F80)
    assert quant.bf16_encode(1.0 + 3 * 2 ** -8) == 0x3F82       # halfway: to even (0x3F82)
    assert quant.bf16_encode(1.0 + 2 ** -8 + 2 ** -20) == 0x3F81
    assert quant.bf16_encode(np.nan) == 0x7FC0
    assert quant.bf16_value(0x4049) == 3.140625
    assert quant.bf16_encode(3.14159265) == 0x4049


def test_e4m3_known_codes():
    assert quant.e4m3_value(0x38) == 1.0
    assert quant.e4m3_value(0x7E) == 448.0
    assert quant.e4m3_value(0x01) == 2.0 ** -9
    assert quant.e4m3_value(0x08) == 2.0 ** -6
    assert quant.e4m3_value(0x07) == 7 / 8 * 2.0 ** -6
    assert np.isnan(quant.e4m3_value(0x7F)) and np.isnan(quant.e4m3_value(0xFF))
    assert quant.e4m3_encode(1.0) == 0x38
    assert quant.e4m3_encode(500.0) == 0x7E and quant.e4m3_encode(-1e9) == 0xFE
    assert quant.e4m3_encode(-0.0) == 0x80
    assert quant.e4m3_encode(1.0625) == 0x38                     # halfway 1.0 / 1.125: even
    assert quant.e4m3_encode(1.1875) == 0x3A                     # halfway 1.125 / 1.25: even
    assert quant.e4m3_encode(2.0 ** -10) == 0x00                 # halfway 0 / min subnormal: even (0)
    assert quant.e4m3_encode(3 * 2.0 ** -10) == 0x02             # halfway 1 / 2 subnormal: even
    assert quant.e4m3_encode(464.0) == 0x7E                      # past 448 saturates


def test_e4m3_round_trip_every_code():
    for c in range(256):
        v = quant.e4m3_value(c)
        if np.isnan(v):
            continue
        assert quant.e4m3_encode(v) == c


def test_scale_and_quantize_error_bound():
    g = np.random.default_rng(0)
    rows = (g.standard_normal((40, 16)) * 3).astype(np.float32)
    s = quant.partition_scale(rows)
    assert s == np.float32(np.abs(rows).max() / np.float32(448))
    codes = quant.quantize_e4m3(rows, s)
    back = quant.dequantize_e4m3(codes, s)
    # E4M3 has 3 fraction bits: relative error <= 2^-4 for normal values
    big = np.abs(rows) > 2 ** -6 * s
    assert np.all(np.abs(back[big] - rows[big]) <= 2 ** -4 * np.abs(rows[big]) + 1e-12)
    assert quant.partition_scale(np.zeros((3, 4), np.float32)) == 1.0
