"""Reduced-precision control-matrix storage, FP64 oracle side -- test infrastructure only.

Sec. 2.3.4 stores the control matrix in 16 bits and widens each value to 32
bits just before the multiply-add, to cut the bytes the bandwidth-bound MVM
moves.  The same idea is applied here with four formats:

* FP16: IEEE binary16, the paper's own 16-bit format, round to nearest even;
* BF16: each FP32 entry rounded to the nearest bfloat16 (8 exponent bits,
  7 stored mantissa bits), ties to even;
* FP8 E4M3 ("fn" variant: bias 7, no infinities, largest finite 448, one NaN
  code) with one FP32 scale per matrix row, ``scale_r = max_j |M_rj| / 448``;
  each code is ``e4m3(M_rj / scale_r)``, rounded to nearest, ties to even,
  saturating at +-448, and the dequantised entry is ``scale_r * code``;
* INT8 with one FP32 scale per row, ``scale_r = max_j |M_rj| / 127``, codes
  ``round_half_even(M_rj / scale_r)`` clamped to [-127, 127], dequantised as
  ``scale_r * code``.  The same bytes as FP8 with a uniform grid of 255 levels
  instead of a 3-bit mantissa: not in the paper, a remedy for the FP8 error.

Quantisation decides an integer code from floating-point arithmetic, so it is
done in IEEE single precision exactly as the device library does it (the
row maximum, the division by 448 and the division by the scale are each one
correctly rounded FP32 operation).  Rounding is written from the formats'
definitions: the E4M3 table below is enumerated from the bit layout.

Parity pins: f16_round, bf16_round and e4m3_round are pinned in
tests/test_oracle_pins.py against brute-force nearest-value search over the
enumerated format and against the independent conversions of libraries (numpy,
torch); the per-row scales by their invariants (the row maximum maps to +-448 or
+-127 exactly) and the INT8 codes by hand-computed ties.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
INT8_MAX = 127.0
F16_MAX = 65504.0


def bf16_round(x):
    """Round FP32 values to the nearest bfloat16 (ties to even); returns float32 values."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    u = (u + 0x7FFF + keep_lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(x32.shape)


def f16_values():
    """All non-negative finite binary16 values in code order 0 .. 0x7BFF."""
    code = np.arange(0x7C00, dtype=np.int64)
    e, m = code >> 10, code & 0x3FF
    sub = (m / 1024.0) * 2.0 ** -14
    nrm = (1.0 + m / 1024.0) * np.power(2.0, (e - 15).astype(np.float64))
    return np.where(e == 0, sub, nrm)


_F16 = f16_values()


def f16_round(x):
    """Round to the nearest binary16 value, ties to the even code; magnitudes at or
    beyond 65520 (half an ulp above the largest finite value) become infinite.
    Returns float64 values."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    hi = np.clip(np.searchsorted(_F16, np.minimum(a, F16_MAX), side="left"), 0, len(_F16) - 1)
    lo = np.clip(hi - 1, 0, len(_F16) - 1)
    dlo = np.minimum(a, F16_MAX) - _F16[lo]
    dhi = _F16[hi] - np.minimum(a, F16_MAX)
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    v = np.where(pick_hi, _F16[hi], _F16[lo])
    v = np.where(a >= 65520.0, np.inf, v)
    return np.sign(x) * v


def e4m3_values():
    """All non-negative finite E4M3 values in code order 0..126 (code 127 is NaN)."""
    vals = []
    for code in range(127):
        e, m = code >> 3, code & 7
        if e == 0:
            vals.append((m / 8.0) * 2.0 ** -6)          # subnormal
        else:
            vals.append((1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals, dtype=np.float64)


_E4M3 = e4m3_values()


def e4m3_round(x):
    """Round to the nearest E4M3 value, ties to the even code, saturating at +-448.

    Returns the rounded values as float64 (exactly representable)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.clip(np.searchsorted(_E4M3, a, side="left"), 0, len(_E4M3) - 1)
    lo = np.clip(hi - 1, 0, len(_E4M3) - 1)
    dlo = a - _E4M3[lo]
    dhi = _E4M3[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo)
    return np.sign(x) * _E4M3[code]


def fp8_row_quantise(M32):
    """Per-row E4M3 quantisation of an FP32 matrix.

    Returns (codes as float64 values, scales float32[nact]); the stored matrix
    is ``scales[:, None] * codes``.  A row of zeros gets scale 1 and zero codes.
    """
    M32 = np.asarray(M32, dtype=np.float32)
    amax = np.max(np.abs(M32), axis=1)
    scale = np.where(amax > 0, amax / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    q = e4m3_round((M32 / scale[:, None]).astype(np.float32))
    return q, scale


def int8_row_quantise(M32):
    """Per-row symmetric INT8 quantisation of an FP32 matrix.

    Returns (codes as float64 integers, scales float32[nact]); the stored matrix is
    ``scales[:, None] * codes``.  Both divisions are single correctly rounded FP32
    operations, the code is the nearest integer (ties to even) of the FP32
    quotient, clamped to [-127, 127].  A row of zeros gets scale 1 and zero codes.
    """
    M32 = np.asarray(M32, dtype=np.float32)
    amax = np.max(np.abs(M32), axis=1)
    scale = np.where(amax > 0, amax / np.float32(INT8_MAX), np.float32(1.0)).astype(np.float32)
    q = np.rint((M32 / scale[:, None]).astype(np.float32).astype(np.float64))
    return np.clip(q, -INT8_MAX, INT8_MAX), scale


def stored_matrix(M32, store):
    """The matrix exactly as the device stores it, in FP64:
    store in {'f32', 'f16', 'bf16', 'fp8', 'int8'}."""
    M32 = np.asarray(M32, dtype=np.float32)
    if store == "f32":
        return M32.astype(np.float64)
    if store == "f16":
        return f16_round(M32)
    if store == "bf16":
        return bf16_round(M32).astype(np.float64)
    if store == "fp8":
        q, sc = fp8_row_quantise(M32)
        return sc.astype(np.float64)[:, None] * q
    if store == "int8":
        q, sc = int8_row_quantise(M32)
        return sc.astype(np.float64)[:, None] * q
    raise ValueError(store)
