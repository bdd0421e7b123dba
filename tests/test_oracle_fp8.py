"""Pins of the oracle's e4m3 decoder (values the format fixes) and of the input quantiser."""
import numpy as np

from oracle import fp8
import synth


def test_e4m3_values_fixed_by_the_format():
    cases = {0x00: 0.0, 0x38: 1.0, 0x3F: 1.875, 0x40: 2.0, 0x7E: 448.0, 0x08: 2.0 ** -6,
             0x01: 2.0 ** -9, 0x07: 7 * 2.0 ** -9, 0xB8: -1.0, 0xFE: -448.0, 0x30: 0.5}
    for code, val in cases.items():
        assert fp8.decode_e4m3([code])[0] == val, hex(code)
    assert np.isnan(fp8.decode_e4m3([0x7F])[0]) and np.isnan(fp8.decode_e4m3([0xFF])[0])
    assert np.signbit(fp8.decode_e4m3([0x80])[0])


def test_positive_codes_are_increasing():
    v = fp8.decode_e4m3(np.arange(0x7F, dtype=np.uint8))
    assert np.all(np.diff(v) > 0)


def test_quantiser_round_trip_within_half_an_ulp():
    X = np.random.default_rng(0).standard_normal((64, 300)) * np.logspace(-3, 3, 64)[:, None]
    codes, scales = synth.quantize_e4m3_rows(X)
    R = fp8.dequantize_rows(codes, scales)
    assert np.all(np.isfinite(R))
    big = np.abs(X) >= 2.0 ** -6 * scales[:, None]   # normal range of e4m3 after scaling
    rel = np.abs(R - X)[big] / np.abs(X)[big]
    assert rel.max() <= 2.0 ** -4 + 1e-12
    np.testing.assert_allclose(np.max(np.abs(R), axis=1), np.max(np.abs(X), axis=1), rtol=1e-6)
