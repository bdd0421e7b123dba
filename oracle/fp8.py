"""FP8 e4m3 decoding for the oracle (test infrastructure only).

The precision form stores minibatch rows as FP8 e4m3 codes with one scale per row:
the value of element (r, c) is scale_r * e4m3(code_rc). This module decodes codes
from the format's definition (1 sign bit, 4 exponent bits with bias 7, 3 mantissa
bits; exponent 0 is subnormal; no infinities; S.1111.111 is NaN), exactly, in
float64. Pins: tests/test_oracle_fp8.py (values fixed by the format).
"""
from __future__ import annotations

import numpy as np


def decode_e4m3(codes) -> np.ndarray:
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 0x7).astype(np.float64)
    normal = sign * np.ldexp(1.0 + m / 8.0, (e - 7).astype(np.int64))
    sub = sign * np.ldexp(m / 8.0, -6)
    out = np.where(e == 0, sub, normal)
    return np.where((e == 15) & ((c & 0x7) == 7), np.nan, out)


def dequantize_rows(codes, scales) -> np.ndarray:
    """Rows scale_r * e4m3(code_r.), in float64."""
    return decode_e4m3(codes) * np.asarray(scales, dtype=np.float64)[:, None]
