"""Pins for the oracle's inspection helpers: the row view (bit `pos` of every
cell of a table) and the per-cell population counts.

Both are the expected-value source of the full-size GPU index checks, so each
is pinned here to something other than itself:

- closed form: one key x inserted into one set i sets, in table r, exactly the
  eta bits h_{r,j}(x) (multiply-shift of Sec. 2's hash, computed here with
  Python integers) of the Bloom filter of cell phi_r(i) (Carter-Wegman,
  Python integers) and nothing else (Algorithm 1, Sec. 3.1);
- consistency with the filter bits themselves: the row view must be the
  transpose of the per-cell filters, and the count must be their popcount,
  over B values whose rows span one word, a ragged word and several words.
"""
import numpy as np
import pytest

P61 = (1 << 61) - 1
M64 = (1 << 64) - 1


def _mix64(z: int) -> int:
    # SplitMix64's output finalizer (Steele, Lea, Flood 2014), Python integers
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _positions(s, r, eta, L, x):
    return sorted({((s[r][j] * _mix64(x)) & M64) >> (64 - L) for j in range(eta)})


def _cell(a, c, r, i, B):
    return ((a[r] * i + c[r]) % P61) % B


def _row_bit(row_words, b):
    return int((int(row_words[b >> 6]) >> (b & 63)) & 1)


@pytest.mark.parametrize("B", [1, 33, 64, 320])
def test_one_key_sets_exactly_its_eta_bits_in_its_cell(oracle_mod, B):
    R, L, eta, K = 3, 12, 3, 400
    m = 1 << L
    o = oracle_mod.Oracle(K, B, R, m, eta, 2024)
    a, c, s = o.params()
    # a set whose cell in some table lies past the first 64-bit word when B > 64
    i = next((t for t in range(K) if B <= 64 or any(_cell(a, c, r, t, B) >= 64 for r in range(R))), 0)
    x = 0x0123456789ABCDEF
    o.insert_keys(i, [x])
    pc = o.cell_popcount()
    rng = np.random.default_rng(B)
    for r in range(R):
        cell = _cell(a, c, r, i, B)
        pos = _positions(s, r, eta, L, x)
        want_pc = np.zeros(B, np.uint64)
        want_pc[cell] = len(pos)
        assert np.array_equal(pc[r], want_pc)
        for p in pos:
            row = o.get_row(r, p)
            assert row.size == (B + 63) // 64
            assert [b for b in range(B) if _row_bit(row, b)] == [cell]
        others = [int(p) for p in rng.integers(0, m, 64) if int(p) not in pos] + [q for q in (0, m - 1) if q not in pos]
        for p in others:
            assert not np.any(o.get_row(r, p))
        # and the filter of that cell, bit by bit
        bits = o.bf_bits(r, cell)
        assert list(np.flatnonzero(bits)) == pos


def test_two_keys_in_two_sets_give_the_union_of_their_rows(oracle_mod):
    B, R, L, eta, K = 96, 2, 10, 2, 500
    o = oracle_mod.Oracle(K, B, R, 1 << L, eta, 7)
    a, c, s = o.params()
    # two sets in different cells of table 0
    i1 = 3
    i2 = next(t for t in range(K) if _cell(a, c, 0, t, B) != _cell(a, c, 0, i1, B))
    x1, x2 = 11, 987654321
    o.insert_keys(i1, [x1])
    o.insert_keys(i2, [x2])
    for r in range(R):
        want = {}
        for i, x in ((i1, x1), (i2, x2)):
            for p in _positions(s, r, eta, L, x):
                want.setdefault(p, set()).add(_cell(a, c, r, i, B))
        for p, cells in want.items():
            row = o.get_row(r, p)
            assert {b for b in range(B) if _row_bit(row, b)} == cells


@pytest.mark.parametrize("B", [1, 33, 64, 320])
def test_row_view_is_the_transpose_of_the_filters(oracle_mod, B):
    R, L, eta, K = 2, 11, 2, 300
    m = 1 << L
    o = oracle_mod.Oracle(K, B, R, m, eta, 99)
    rng = np.random.default_rng(B + 1)
    for i in range(0, K, 3):
        o.insert_keys(i, rng.integers(0, 1 << 62, 20, dtype=np.uint64))
    for r in range(R):
        bits = np.stack([o.bf_bits(r, b) for b in range(B)])  # [B][m]
        for p in list(rng.integers(0, m, 200)) + [0, m - 1]:
            row = o.get_row(r, int(p))
            got = np.array([_row_bit(row, b) for b in range(B)], np.uint8)
            assert np.array_equal(got, bits[:, int(p)])
            # bits past B in the last word stay zero
            if B % 64:
                assert int(row[-1]) >> (B % 64) == 0


@pytest.mark.parametrize("B", [1, 33, 320])
def test_cell_popcount_equals_the_filters_set_bits(oracle_mod, B):
    R, L, eta, K = 3, 12, 3, 400
    o = oracle_mod.Oracle(K, B, R, 1 << L, eta, 5)
    rng = np.random.default_rng(B + 2)
    for i in range(0, K, 2):
        o.insert_keys(i, rng.integers(0, 1 << 62, 15, dtype=np.uint64))
    pc = o.cell_popcount()
    for r in range(R):
        for b in range(B):
            w = o.export_bf(r, b)
            assert int(pc[r, b]) == int(np.unpackbits(w.view(np.uint8)).sum())
