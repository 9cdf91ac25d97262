"""Plain definitions of the storage roundings (test infrastructure only).

The gridding path can store spectra as BF16 or as FP8 e4m3 with a
per-channel scale.  These are the definitions the CUDA ingest must match bit
for bit:

* BF16: round-to-nearest, ties to even, of the FP32 value to 8 significant
  bits (the upper half of the FP32 bit pattern).
* E4M3 ("fn" variant: bias 7, no infinities, 0x7F/0xFF are NaN, largest
  finite value 448): per channel c the scale is ``s_c = amax_c / 448`` in FP32,
  where amax_c is the largest finite |x| of the channel (``s_c = 1`` when
  amax_c is 0), the scaled value is ``y = x / s_c`` in FP32, and the code is
  the e4m3 value nearest to y, ties to the even code, with |y| beyond 448
  saturating to +-448 and NaN mapping to NaN.

The paper itself stores no reduced precision; these readings come from the
mixed-precision form of the method and are this package's choices, not the
paper's.
"""
from __future__ import annotations

import numpy as np


def bf16_round_bits(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest even."""
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    r = np.where(nan, ((u >> 16) | 0x40).astype(np.uint16), r)   # keep NaN quiet
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


def e4m3_table() -> np.ndarray:
    """Values of the codes 0x00..0x7E (all finite non-negative e4m3 values)."""
    vals = np.empty(127, np.float64)
    for code in range(127):
        e = (code >> 3) & 0xF
        m = code & 0x7
        vals[code] = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


_E4 = e4m3_table()


def e4m3_encode(y: np.ndarray) -> np.ndarray:
    """FP32 values -> e4m3 codes (uint8): nearest, ties to even, saturating."""
    y = np.asarray(y, np.float32).astype(np.float64).ravel()
    a = np.minimum(np.abs(y), 448.0)
    hi = np.searchsorted(_E4, a, side="left")          # first table value >= a
    hi = np.minimum(hi, 126)
    lo = np.maximum(hi - 1, 0)
    dlo = a - _E4[lo]
    dhi = _E4[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo)
    code = np.where(a == _E4[hi], hi, code)             # exact values
    sign = np.signbit(y).astype(np.int64) << 7
    out = (code | sign).astype(np.uint8)
    out = np.where(np.isnan(y), np.uint8(0x7F), out)
    return out.astype(np.uint8)


def e4m3_decode(code: np.ndarray) -> np.ndarray:
    c = np.asarray(code, np.uint8).astype(np.int64)
    mag = c & 0x7F
    v = np.where(mag == 0x7F, np.nan, _E4[np.minimum(mag, 126)])
    return np.where(c & 0x80, -v, v)


def e4m3_scales(x: np.ndarray) -> np.ndarray:
    """Per-channel FP32 scales s_c = amax_c / 448 of x[N, C] (1 for amax 0)."""
    x = np.asarray(x, np.float32)
    ax = np.where(np.isfinite(x), np.abs(x), np.float32(0))
    amax = ax.max(axis=0) if x.shape[0] else np.zeros(x.shape[1], np.float32)
    amax = amax.astype(np.float32)
    s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    return s


def e4m3_quantise(x: np.ndarray):
    """x[N, C] FP32 -> (codes uint8 [N, C], scales float32 [C])."""
    x = np.asarray(x, np.float32)
    s = e4m3_scales(x)
    y = (x / s[None, :]).astype(np.float32)
    return e4m3_encode(y).reshape(x.shape), s


def e4m3_dequantise(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """Dequantised values in FP64: decode(code) * scale (exact in FP64)."""
    return e4m3_decode(codes) * np.asarray(scales, np.float32).astype(np.float64)[None, :]
