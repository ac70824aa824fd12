"""Low-precision storage formats (oracle; test infrastructure only).

The index can store base vectors in BF16, or in FP8 E4M3 with a scale per
partition (a compressed form of the partitions the paper names as future
work, Sec. 9), scan them with FP32 accumulation and re-rank an oversized
candidate list exactly in FP32.  This module restates the two formats from
their definitions, by brute force:

  BF16   the upper 16 bits of an IEEE binary32: 1 sign, 8 exponent, 7 fraction
         bits.  FP32 -> BF16 rounds to the nearest representable value, ties
         to the even fraction; NaN becomes the quiet NaN 0x7FC0.
  E4M3   OCP 8-bit floating point E4M3: 1 sign, 4 exponent bits (bias 7), 3
         fraction bits; exponent field 0 holds subnormals m/8 * 2^-6; the
         all-ones pattern S.1111.111 is NaN; there is no infinity; the
         largest finite magnitude is 448 = 1.75 * 2^8.  FP32 -> E4M3 rounds to
         the nearest finite value, ties to the even code, and saturates beyond
         +-448; NaN becomes 0x7F.
  scale  per partition, s = max|x| / 448 computed in FP32 (1 if the partition
         is all zero); a row is stored as E4M3(x / s) with the division in FP32
         and read back as decode(code) * s.
"""

import numpy as np


def bf16_value(code):
    """Value of a BF16 bit pattern (as float64)."""
    return float(np.array([int(code) << 16], dtype=np.uint32).view(np.float32)[0])


def _bf16_candidates(x):
    """The two BF16 patterns that bracket the float32 x (same sign)."""
    b = int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    lo = b >> 16
    return lo, lo + 1


def bf16_encode(x):
    """Nearest BF16 to the float32 x, ties to even (brute force over the two neighbours)."""
    x = np.float32(x)
    if np.isnan(x):
        return 0x7FC0
    lo, hi = _bf16_candidates(x)
    vx = float(x)
    vlo, vhi = bf16_value(lo), bf16_value(hi & 0xFFFF) if (hi & 0xFFFF) == hi else float("inf")
    dlo, dhi = abs(vx - vlo), abs(vhi - vx)
    if dlo < dhi:
        return lo
    if dhi < dlo:
        return hi & 0xFFFF
    return lo if lo % 2 == 0 else hi & 0xFFFF


def e4m3_value(code):
    """Value of an E4M3 code (NaN for S.1111.111)."""
    code = int(code) & 0xFF
    sign = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return sign * (m / 8.0) * 2.0 ** -6
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


_POS_CODES = np.array([c for c in range(0x7F)], dtype=np.int64)          # +0 .. 448
_POS_VALS = np.array([e4m3_value(c) for c in _POS_CODES])


def e4m3_encode(x):
    """Nearest finite E4M3 to x (ties to the even code), saturating at +-448."""
    x = float(x)
    if np.isnan(x):
        return 0x7F
    sign = 0x80 if (x < 0 or (x == 0 and np.signbit(x))) else 0
    a = abs(x)
    d = np.abs(_POS_VALS - a)
    best = np.nonzero(d == d.min())[0]
    code = int(_POS_CODES[best[0]])
    if len(best) > 1:                       # a tie: take the even code
        even = [int(_POS_CODES[b]) for b in best if _POS_CODES[b] % 2 == 0]
        code = even[0]
    return sign | code


def partition_scale(rows):
    """s = max|x| / 448 in FP32 (1 for an all-zero partition)."""
    rows = np.asarray(rows, dtype=np.float32)
    if rows.size == 0:
        return np.float32(1.0)
    m = np.float32(np.abs(rows).max())
    if m == 0:
        return np.float32(1.0)
    return np.float32(m / np.float32(448.0))


def quantize_e4m3(rows, scale):
    """E4M3 codes of rows / scale (division in FP32)."""
    rows = np.asarray(rows, dtype=np.float32)
    y = (rows / np.float32(scale)).astype(np.float32)
    out = np.empty(y.shape, dtype=np.uint8)
    flat = y.reshape(-1)
    o = out.reshape(-1)
    cache = {}
    for i, v in enumerate(flat):
        key = v.tobytes()
        c = cache.get(key)
        if c is None:
            c = e4m3_encode(v)
            cache[key] = c
        o[i] = c
    return out


def quantize_bf16(rows):
    rows = np.asarray(rows, dtype=np.float32)
    out = np.empty(rows.shape, dtype=np.uint16)
    flat, o = rows.reshape(-1), out.reshape(-1)
    for i, v in enumerate(flat):
        o[i] = bf16_encode(v)
    return out


def dequantize_e4m3(codes, scale):
    table = np.array([e4m3_value(c) for c in range(256)])
    return (table[np.asarray(codes, dtype=np.int64)] * np.float64(scale)).astype(np.float64)


def dequantize_bf16(codes):
    return np.asarray(codes, dtype=np.uint32).__lshift__(16).astype(np.uint32).view(np.float32).astype(np.float64)
