"""Reduced-precision storage of Q for the oracle -- test infrastructure only.

The paper states no storage precision.  These functions define, from the
number formats' published definitions, the quantised matrices that the mixed
precision path stores, so that the oracle can solve exactly the quantised
problem and the codes can be compared bit for bit:

  * bfloat16: the top 16 bits of an IEEE binary32 value after rounding the
    dropped 16 bits to nearest, ties to even.
  * FP8 E4M3 (OCP 8-bit floating point, "E4M3FN"): sign, 4 exponent bits with
    bias 7, 3 mantissa bits; exponent field 0 holds subnormals m/8 * 2^-6;
    no infinities; S.1111.111 is NaN, so the largest finite value is
    1.75 * 2^8 = 448.  Conversion rounds to nearest, ties to even, and
    saturates finite out-of-range values to +-448.
  * Symmetric Jacobi-scaled FP8 storage: r_j = 1/sqrt(Q_jj) (1 when Q_jj <= 0),
    C_jk = ((Q_jk * r_j) * r_k) * 256 in float32, codes = E4M3(C), and
    s'_j = sqrt(Q_jj) / 16 (1/16 when Q_jj <= 0), so the stored matrix is
    Q~_jk = s'_j * dec(code_jk) * s'_k.  For PSD Q, |C_jk| <= 256 < 448.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (returned as float32 holding the bf16 value)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(x)
    out[nan] = np.nan
    return out


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def e4m3_decode_table() -> np.ndarray:
    """float64 value of each of the 256 E4M3 codes (NaN for the two NaN codes)."""
    vals = np.empty(256, np.float64)
    for code in range(256):
        s = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        mnt = code & 0x7
        if e == 0xF and mnt == 0x7:
            vals[code] = np.nan
        elif e == 0:
            vals[code] = s * (mnt / 8.0) * 2.0 ** (-6)
        else:
            vals[code] = s * (1.0 + mnt / 8.0) * 2.0 ** (e - 7)
    return vals


_TABLE = e4m3_decode_table()
_POS_CODES = np.arange(0, 0x7F)            # 0x00 .. 0x7E: all finite non-negative values
_POS_VALS = _TABLE[_POS_CODES]             # ascending


def e4m3_encode(x: np.ndarray) -> np.ndarray:
    """uint8 E4M3 codes of float32 x: nearest value, ties to the even code,
    finite out-of-range saturated to +-448, NaN -> 0x7F."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.abs(x)
    idx = np.searchsorted(_POS_VALS, a, side="left")      # first value >= a
    idx = np.clip(idx, 1, len(_POS_VALS) - 1)
    lo, hi = _POS_VALS[idx - 1], _POS_VALS[idx]
    dlo, dhi = a - lo, hi - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((_POS_CODES[idx] & 1) == 0))
    code = np.where(pick_hi, _POS_CODES[idx], _POS_CODES[idx - 1])
    code = np.where(a <= 0.0, 0, code)
    code = np.where(a >= _POS_VALS[-1], 0x7E, code)       # saturate (satfinite)
    code = code.astype(np.uint8) | np.where(np.signbit(x), 0x80, 0).astype(np.uint8)
    code = np.where(np.isnan(x), 0x7F, code).astype(np.uint8)
    return code


def e4m3_round(x: np.ndarray) -> np.ndarray:
    """Value (float64) of the E4M3 code nearest to x."""
    return _TABLE[e4m3_encode(x)]


def fp8_jacobi_quantize(Q: np.ndarray):
    """Symmetric Jacobi-scaled E4M3 storage of one symmetric float32 matrix.

    Returns (codes uint8 (n, n), s float32 (n,)) with Q~ = diag(s) dec(codes) diag(s).
    """
    Q = np.asarray(Q, dtype=np.float32)
    dg = np.diagonal(Q).astype(np.float32)
    pos = dg > 0
    sq = np.where(pos, np.sqrt(np.where(pos, dg, np.float32(1))), np.float32(1)).astype(np.float32)
    r = (np.float32(1) / sq).astype(np.float32)
    # Q_jk * (r_j * r_k): the product of the two factors first, so that the
    # codes of (j, k) and (k, j) are equal and Q~ is exactly symmetric
    rr = (r[:, None] * r[None, :]).astype(np.float32)
    C = (Q * rr).astype(np.float32)
    C = (C * np.float32(256.0)).astype(np.float32)
    codes = e4m3_encode(C)
    s = (sq * np.float32(1.0 / 16.0)).astype(np.float32)
    return codes, s


def fp8_dequantize(codes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """float64 Q~ = diag(s) dec(codes) diag(s)."""
    s64 = np.asarray(s, np.float64)
    return s64[:, None] * _TABLE[codes] * s64[None, :]


def jacobi_factors(diag: np.ndarray):
    """(r, s') of the symmetric Jacobi-scaled storage from the float32 diagonal:
    r_j = 1/sqrt(Q_jj), s'_j = sqrt(Q_jj)/16 (r_j = 1, s'_j = 1/16 when Q_jj <= 0)."""
    dg = np.asarray(diag, dtype=np.float32)
    pos = dg > 0
    sq = np.where(pos, np.sqrt(np.where(pos, dg, np.float32(1))), np.float32(1)).astype(np.float32)
    r = (np.float32(1) / sq).astype(np.float32)
    return r, (sq * np.float32(1.0 / 16.0)).astype(np.float32)


def fp8_jacobi_codes(q: np.ndarray, r_row: np.ndarray, r_col: np.ndarray) -> np.ndarray:
    """E4M3 codes of single entries Q_jk of the Jacobi-scaled storage, given
    r_j and r_k (broadcast against q): E4M3((Q_jk * (r_j * r_k)) * 256), each
    product rounded to float32 as in fp8_jacobi_quantize.  Lets a few rows or
    columns of a matrix too large to quantise here be checked on their own."""
    q = np.asarray(q, dtype=np.float32)
    rr = (np.asarray(r_row, np.float32) * np.asarray(r_col, np.float32)).astype(np.float32)
    C = (q * rr).astype(np.float32)
    return e4m3_encode((C * np.float32(256.0)).astype(np.float32))
