"""The right-hand-side pieces of the tensor-core tile products, checked on the
host: the quantised tiles are multiplied, on the tensor cores, by pieces of
the tile's own type that add up to the float32 right-hand side, so that every
product of a code and a piece is exact and only the float32 accumulation
rounds.  These tests pin the splitting scheme the kernel follows (one
128-entry slice at a time), with float32 arithmetic as on the device and the
bit-level BF16 / E4M3 roundings of the oracle's quantisers:

* BF16: e = h + m + l with h = rn(e), m = rn(e - h), l = rn(e - h - m): exact
  (three times 8 significant bits, each subtraction exact) for |e| >= 2^-100;
  below that the last piece can be a bf16 subnormal (error under 2^-133);
* FP8: a power of two sigma per slice with |sigma e| < 256, then six e4m3
  pieces, each residual scaled by 16 before it is rounded: sigma e = sum_j
  q_j 16^-j to 2^-23 of each entry or 2^-37 of the slice's largest entry,
  whichever is larger; no piece saturates, every subtraction and scaling is
  exact; an all-zero slice gives zero pieces.
"""
import math

import numpy as np
import pytest

from oracle import quant as Qz

F32 = np.float32


def split_bf16(e):
    e = e.astype(F32)
    pieces, a = [], e.copy()
    for _ in range(3):
        q = Qz.bf16_round(a)
        pieces.append(q)
        nxt = (a - q).astype(F32)
        assert np.array_equal(nxt.astype(np.float64), a.astype(np.float64) - q.astype(np.float64))   # exact
        a = nxt
    return pieces, a


def split_e4m3(e):
    """One slice: (1 / sigma, six pieces, the dropped residual in sigma units)."""
    e = e.astype(F32)
    mx = float(np.max(np.abs(e))) if e.size else 0.0
    _, ex = math.frexp(mx)                       # mx < 2^ex (ex = 0 for mx = 0)
    ex = max(-100, min(ex, 100))
    sig, isig = F32(2.0 ** (8 - ex)), F32(2.0 ** (ex - 8))
    a = (e * sig).astype(F32)
    assert np.all(np.abs(a) < 256)
    pieces = []
    for j in range(6):
        q = Qz.e4m3_round(a).astype(F32)
        assert np.all(np.abs(q) <= 448)          # never saturates
        nxt = ((a - q) * F32(16)).astype(F32)
        assert np.array_equal(nxt.astype(np.float64), (a.astype(np.float64) - q.astype(np.float64)) * 16)
        pieces.append(q)
        a = nxt
    return isig, pieces, a


def slices(rng, n_slices):
    """Float32 slices of very different magnitudes, one all zero."""
    out = []
    for k in range(n_slices):
        scale = 10.0 ** rng.uniform(-30, 30)
        v = (rng.standard_normal(128) * scale).astype(F32)
        v[rng.random(128) < 0.1] = 0.0
        v[rng.random(128) < 0.05] *= F32(1e-6)    # small entries beside large ones
        out.append(v)
    out.append(np.zeros(128, F32))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_bf16_pieces_are_exact(seed):
    rng = np.random.default_rng(seed)
    for e in slices(rng, 16):
        pieces, rest = split_bf16(e)
        total = sum(p.astype(np.float64) for p in pieces)
        e64 = e.astype(np.float64)
        big = np.abs(e64) >= 2.0 ** -100
        assert np.all(rest[big] == 0) and np.array_equal(total[big], e64[big])
        assert np.all(np.abs(total - e64) <= 2.0 ** -133)
        for p in pieces:
            assert np.array_equal(Qz.bf16_round(p), p)     # representable in bf16


@pytest.mark.parametrize("seed", range(4))
def test_e4m3_pieces_hold_the_slice_to_float32_accuracy(seed):
    rng = np.random.default_rng(100 + seed)
    for e in slices(rng, 16):
        isig, pieces, rest = split_e4m3(e)
        recon = sum(p.astype(np.float64) * 16.0 ** (-j) for j, p in enumerate(pieces)) * float(isig)
        e64 = e.astype(np.float64)
        mx = float(np.max(np.abs(e64)))
        # the dropped residual is at most half an e4m3 step of the last piece:
        # 2^-24 of the entry while the pieces stay normal, else half the
        # subnormal step of the sixth piece, 2^-10 16^-5 in units of sigma
        # (|sigma e| < 2^8): 2^-38 of the slice's largest entry
        err = np.abs(recon - e64)
        assert np.all(err <= 2.0 ** -23 * np.abs(e64) + 2.0 ** -37 * mx), (err.max(), mx)
        for p in pieces:
            assert np.array_equal(Qz.e4m3_round(p).astype(F32), p)    # representable in e4m3
        if mx == 0.0:
            assert all(np.all(p == 0) for p in pieces) and isig == F32(2.0 ** -8)


def test_e4m3_pieces_products_are_exact_in_float32():
    """Every code x piece product (4 x 4 significant bits) and every bf16 x bf16
    product (8 x 8) is exact in float32, so only the accumulation rounds."""
    codes = Qz.e4m3_decode_table()
    codes = codes[np.isfinite(codes)]
    prod = np.outer(codes, codes)
    assert np.array_equal(prod.astype(F32).astype(np.float64), prod)
    rng = np.random.default_rng(9)
    a = Qz.bf16_round(rng.standard_normal(4000).astype(F32)).astype(np.float64)
    b = Qz.bf16_round(rng.standard_normal(4000).astype(F32)).astype(np.float64)
    assert np.array_equal((a * b).astype(F32).astype(np.float64), a * b)
