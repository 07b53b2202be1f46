"""Pins of the oracle's storage quantisers to the number formats' definitions.

bfloat16 and FP8 E4M3 are fixed by their published formats; PyTorch's CPU
conversions to ``torch.bfloat16`` and ``torch.float8_e4m3fn`` (round to
nearest even) are an independent implementation of the same definitions.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import quant as QZ


def test_bf16_matches_torch_and_is_rne():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.4e38], np.float32)])
    ours = QZ.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours.view(np.uint32), ref.view(np.uint32))
    # ties: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even mantissa (1.0)
    assert QZ.bf16_round(np.array([1.0 + 2.0 ** -8], np.float32))[0] == 1.0
    assert QZ.bf16_round(np.array([1.0 + 3 * 2.0 ** -8], np.float32))[0] == 1.0 + 2.0 ** -6


def test_e4m3_table_special_values():
    t = O.e4m3_decode_table()
    assert t[0x7E] == 448.0 and t[0xFE] == -448.0          # largest finite
    assert t[0x01] == 2.0 ** -9                            # smallest subnormal
    assert t[0x08] == 2.0 ** -6                            # smallest normal
    assert t[0x38] == 1.0                                  # exponent field 7 = bias
    assert np.isnan(t[0x7F]) and np.isnan(t[0xFF])
    finite = t[np.isfinite(t)]
    assert len(finite) == 254


def test_e4m3_encode_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-500, 500, 5000), rng.standard_normal(5000) * 1e-2,
                        rng.standard_normal(5000)]).astype(np.float32)
    codes = QZ.e4m3_encode(x)
    ref_vals = torch.from_numpy(np.clip(x, -448, 448)).to(torch.float8_e4m3fn)
    ref_codes = ref_vals.view(torch.uint8).numpy()
    # torch maps -0 results to 0x80; compare values, not signed-zero codes
    ours = O.e4m3_decode_table()[codes]
    theirs = O.e4m3_decode_table()[ref_codes]
    np.testing.assert_array_equal(ours, theirs)
    # saturation of finite out-of-range values
    assert QZ.e4m3_encode(np.array([1e6, -1e6], np.float32)).tolist() == [0x7E, 0xFE]


@pytest.mark.parametrize("seed", range(3))
def test_fp8_jacobi_is_symmetric_and_close(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((40, 64))
    Q = (A.T @ A / 64).astype(np.float32)
    Q = ((Q + Q.T) * np.float32(0.5)).astype(np.float32)
    codes, s = O.fp8_jacobi_quantize(Q)
    Qt = QZ.fp8_dequantize(codes, s)
    np.testing.assert_array_equal(Qt, Qt.T)
    # |scaled entries| <= 256 for PSD Q (correlation-matrix bound), so every
    # code is finite and the relative error is within the 3-bit mantissa
    dec = O.e4m3_decode_table()[codes]
    assert np.all(np.abs(dec) <= 256.0)
    d = np.sqrt(np.diag(Q).astype(np.float64))
    err = np.abs(Qt - Q) / np.outer(d, d)
    assert err.max() <= 2.0 ** -4 + 2.0 ** -9


def test_fp8_codes_are_symmetric_near_rounding_ties():
    """The code of (j, k) equals the code of (k, j) even where the scaled
    entry lies next to a tie between two E4M3 values: entries are placed at
    the midpoints of adjacent codes, nudged by one float32 ulp either way, so
    that forming (Q_jk r_j) r_k and (Q_jk r_k) r_j in float32 would round to
    different codes for some of them."""
    rng = np.random.default_rng(12)
    vals = O.e4m3_decode_table()
    pos = np.unique(vals[np.isfinite(vals) & (vals > 0) & (vals <= 256)])
    mids = 0.5 * (pos[:-1] + pos[1:])
    N = 200000
    t = rng.choice(mids, N) * rng.choice([-1.0, 1.0], N)
    rj = rng.uniform(0.3, 3.0, N).astype(np.float32)
    rk = rng.uniform(0.3, 3.0, N).astype(np.float32)
    q = (t / (256.0 * rj.astype(np.float64) * rk)).astype(np.float32)
    q = np.where(rng.random(N) < 0.5, np.nextafter(q, np.float32(np.inf)), np.nextafter(q, np.float32(-np.inf)))
    a = QZ.fp8_jacobi_codes(q, rj, rk)
    b = QZ.fp8_jacobi_codes(q, rk, rj)
    np.testing.assert_array_equal(a, b)
    # the other order of the products does break the symmetry on these entries
    left = ((q * rj).astype(np.float32) * rk).astype(np.float32)
    right = ((q * rk).astype(np.float32) * rj).astype(np.float32)
    e1 = QZ.e4m3_encode((left * np.float32(256)).astype(np.float32))
    e2 = QZ.e4m3_encode((right * np.float32(256)).astype(np.float32))
    assert np.any(e1 != e2)


@pytest.mark.parametrize("seed", range(3))
def test_fp8_entrywise_codes_equal_the_whole_matrix_quantiser(seed):
    """Codes of sampled rows and of single columns, computed entry by entry,
    are the whole-matrix quantiser's codes; a zero-diagonal coordinate (the
    epigraph variable of the kernel-learning form) takes r = 1, s' = 1/16."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((30, 50))
    Q = np.zeros((51, 51), np.float32)
    Q[:50, :50] = A.T @ A / 50
    Q = ((Q + Q.T) * np.float32(0.5)).astype(np.float32)
    codes, s = O.fp8_jacobi_quantize(Q)
    r, s2 = QZ.jacobi_factors(np.diagonal(Q))
    np.testing.assert_array_equal(s2, s)
    assert r[50] == 1.0 and s2[50] == np.float32(1.0 / 16.0)
    rows = np.array([0, 7, 49, 50])
    np.testing.assert_array_equal(QZ.fp8_jacobi_codes(Q[rows], r[rows][:, None], r[None, :]), codes[rows])
    for k in (0, 13, 50):
        np.testing.assert_array_equal(QZ.fp8_jacobi_codes(Q[:, k], r, r[k]), codes[:, k])
