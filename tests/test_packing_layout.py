"""The layout of the symmetric block packing, checked on the CPU against plain
linear algebra (no GPU, no library call):

* tile (I, J), I <= J, of the upper block triangle sits at index
  I T - I (I - 1) / 2 + (J - I), the row-major order of the tile table;
* the slot decomposition: tile (I, J) puts B v_J in slot J of the rows of
  block I and, off the diagonal, B' v_I in slot I of the rows of block J;
  every (row block, slot) pair is written exactly once and the slot sums
  are Q v (float64, exact up to rounding), including a ragged last block;
* the lane-to-row map of the halving reduction over 32 lanes (8 rows per
  warp): each row is held by four lanes, and the halving steps sum the 32
  lanes' partials.
"""
import numpy as np
import pytest

STB = 128


def tile_index(I, J, T):
    return I * T - I * (I - 1) // 2 + (J - I)


def tile_table(T):
    return [(I, J) for I in range(T) for J in range(I, T)]


@pytest.mark.parametrize("T", [1, 2, 3, 8, 32])
def test_tile_index_is_the_row_major_table_order(T):
    table = tile_table(T)
    assert len(table) == T * (T + 1) // 2
    for k, (I, J) in enumerate(table):
        assert tile_index(I, J, T) == k


@pytest.mark.parametrize("n", [100, 128, 129, 300])
def test_slot_decomposition_sums_to_q_v(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    Q = A + A.T
    v = rng.standard_normal(n)
    T = (n + STB - 1) // STB
    Qp = np.zeros((T * STB, T * STB))
    Qp[:n, :n] = Q
    vp = np.zeros(T * STB)
    vp[:n] = v
    ldp = T * STB
    P = np.full((T, ldp), np.nan)        # slot s of row r
    writes = np.zeros((T, T), dtype=int)  # (row block, slot)
    for I, J in tile_table(T):
        B = Qp[I * STB:(I + 1) * STB, J * STB:(J + 1) * STB]   # only the upper triangle is read
        P[J, I * STB:(I + 1) * STB] = B @ vp[J * STB:(J + 1) * STB]
        writes[I, J] += 1
        if I != J:
            P[I, J * STB:(J + 1) * STB] = B.T @ vp[I * STB:(I + 1) * STB]
            writes[J, I] += 1
    assert np.all(writes == 1)
    assert not np.isnan(P).any()
    w = P.sum(axis=0)[:n]
    np.testing.assert_allclose(w, Q @ v, rtol=0, atol=1e-12 * (np.abs(Q) @ np.abs(v)).max())


def halving_rows(a):
    """The halving reduction of 8 row partials over 32 lanes: at step o the
    lanes with bit o set keep the upper half of their rows and add their
    partner's copy; then bits 1 and 0 are summed plainly."""
    a = a.copy()
    h, o = 4, 16
    while h >= 1:
        new = a.copy()
        for lane in range(32):
            p = lane ^ o
            hi = bool(lane & o)
            for k in range(h):
                send = a[p, k] if (p & o) else a[p, k + h]
                keep = a[lane, k + h] if hi else a[lane, k]
                new[lane, k] = keep + send
        a = new
        h >>= 1
        o >>= 1
    r = np.array([a[lane, 0] + a[lane ^ 2, 0] for lane in range(32)])
    return np.array([r[lane] + r[lane ^ 1] for lane in range(32)])


def row_of_lane(lane):
    return 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1)


def test_halving_reduction_lane_to_row_map():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((32, 8))
    out = halving_rows(a)
    sums = a.sum(axis=0)
    counts = np.zeros(8, dtype=int)
    for lane in range(32):
        assert abs(out[lane] - sums[row_of_lane(lane)]) <= 1e-12
        counts[row_of_lane(lane)] += 1
    assert np.all(counts == 4)
    # the writing lanes (lane % 4 == 0) cover the 8 rows once
    assert sorted(row_of_lane(lane) for lane in range(0, 32, 4)) == list(range(8))
