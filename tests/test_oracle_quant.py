"""Pins of the storage-rounding definitions against library conversions and
exhaustive code tables."""
import numpy as np
import torch

from oracle import quant as Q


def test_bf16_matches_torch_rounding():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 200000), rng.uniform(-1e-30, 1e-30, 1000),
                        [0.0, -0.0, 1.0, 65504.0, 3.4e38, -3.4e38, 1e-45]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(Q.bf16_round_bits(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even pattern (1.0)
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8], np.float32)
    out = Q.bf16_bits_to_f32(Q.bf16_round_bits(x))
    assert out[0] == 1.0 and out[1] == 1 + 2 * 2.0 ** -7


def test_e4m3_table_and_roundtrip():
    t = Q.e4m3_table()
    assert t[0] == 0 and t[1] == 2.0 ** -9 and t[8] == 2.0 ** -6 and t[126] == 448.0
    assert np.all(np.diff(t) > 0)
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)
    vals = Q.e4m3_decode(codes).astype(np.float32)
    back = Q.e4m3_encode(vals)
    # -0 encodes back to 0x80, +0 to 0x00
    assert np.array_equal(back, codes)


def test_e4m3_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 200000), rng.normal(0, 0.01, 20000)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(Q.e4m3_encode(x), ref)


def test_e4m3_ties_saturation_nan():
    # halfway between 1.0 (m=0) and 1.125 (m=1) -> even code (1.0)
    assert Q.e4m3_decode(Q.e4m3_encode(np.array([1.0625], np.float32)))[0] == 1.0
    assert Q.e4m3_decode(Q.e4m3_encode(np.array([1.1875], np.float32)))[0] == 1.25
    assert Q.e4m3_decode(Q.e4m3_encode(np.array([1e6, -500.0], np.float32))).tolist() == [448.0, -448.0]
    assert Q.e4m3_encode(np.array([np.nan], np.float32))[0] == 0x7F


def test_e4m3_scales():
    x = np.array([[1.0, -896.0, 0.0], [-3.0, 2.0, 0.0]], np.float32)
    s = Q.e4m3_scales(x)
    assert s.tolist() == [np.float32(3.0) / np.float32(448.0), 2.0, 1.0]
    codes, s2 = Q.e4m3_quantise(x)
    deq = Q.e4m3_dequantise(codes, s2)
    # the channel maximum maps to code 448 exactly; the scale itself is rounded to FP32
    assert deq[1, 0] == -448.0 * float(s2[0]) and deq[0, 1] == -896.0
    assert abs(deq[1, 0] + 3.0) < 3e-7
