"""Pins for the oracle's hash and encoding layer.

The paper asks for eta universal hashes for Bloom-filter positions (Sec. 2) and
R 2-universal partition hashes on set identity (Sec. 3, Fig. 1 caption); the
concrete family is this project's choice (SplitMix64 parameters,
Carter-Wegman phi mod 2^61-1, multiply-shift positions).  Each check compares
the oracle with something other than itself: published generator outputs,
Python's arbitrary-precision arithmetic, closed forms, or statistics.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P61 = (1 << 61) - 1
M64 = (1 << 64) - 1


def _golden_hex(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    return vals


def test_splitmix64_published_outputs(oracle_mod):
    want = _golden_hex("splitmix64_seed0.txt")
    assert oracle_mod.splitmix64_stream(0, len(want)) == want


def test_mix64_fixed_point_and_bijection(oracle_mod):
    # 0 is a fixed point of the xor-shift-multiply finalizer (every step maps 0 to 0)
    assert oracle_mod.mix64(0) == 0
    xs = list(range(1, 20001)) + [1 << s for s in range(64)]
    ys = {oracle_mod.mix64(x) for x in xs}
    assert len(ys) == len(set(xs))  # no collisions: the finalizer is a bijection


def test_params_follow_the_generator_stream(oracle_mod):
    K, B, R, m, eta, seed = 50, 7, 4, 1 << 12, 3, 12345
    o = oracle_mod.Oracle(K, B, R, m, eta, seed)
    a, c, s = o.params()
    stream = oracle_mod.splitmix64_stream(seed, 2 * R + R * eta)
    for r in range(R):
        assert a[r] == 1 + stream[2 * r] % (P61 - 1)
        assert c[r] == stream[2 * r + 1] % P61
        assert 1 <= a[r] < P61 and 0 <= c[r] < P61
    for r in range(R):
        for j in range(eta):
            assert s[r][j] == stream[2 * R + r * eta + j] | 1
            assert s[r][j] & 1


def test_phi_matches_bigint_carter_wegman(oracle_mod):
    B, R = 320, 8
    o = oracle_mod.Oracle(5000, B, R, 1 << 6, 1, 777)
    a, c, _ = o.params()
    rng = np.random.default_rng(0)
    ids = [0, 1, 2, 4999] + [int(v) for v in rng.integers(0, 5000, 500)]
    for r in range(R):
        for i in ids:
            assert o.phi(r, i) == ((a[r] * i + c[r]) % P61) % B
    # IDs near 2^32 exercise the 128-bit product (phi itself takes any 64-bit ID)
    for r in range(R):
        for i in [(1 << 32) - 1, (1 << 32) - 12345, (1 << 31) + 7]:
            assert o.phi(r, i) == ((a[r] * i + c[r]) % P61) % B


def test_phi_two_universal_collision_rate(oracle_mod):
    B, R, K = 16, 6, 4000
    o = oracle_mod.Oracle(K, B, R, 1 << 6, 1, 99)
    tab = o.phi_table()
    rng = np.random.default_rng(1)
    i = rng.integers(0, K, 20000)
    j = rng.integers(0, K, 20000)
    keep = i != j
    coll = (tab[i[keep]] == tab[j[keep]]).mean(axis=0)  # per table
    # each table's collision rate is ~1/B; 4 sigma binomial band per table
    n = keep.sum()
    sd = np.sqrt((1 / B) * (1 - 1 / B) / n)
    assert np.all(np.abs(coll - 1 / B) < 4 * sd + 0.002)
    # cells of one table partition the IDs: every ID has exactly one cell
    assert tab.min() >= 0 and tab.max() < B


def test_positions_match_bigint_multiply_shift(oracle_mod):
    m = 1 << 27
    L = 27
    o = oracle_mod.Oracle(10, 4, 3, m, 2, 2024)
    _, _, s = o.params()
    rng = np.random.default_rng(2)
    keys = [0, 1, M64, (1 << 62) - 1] + [int(v) for v in rng.integers(0, 1 << 62, 300, dtype=np.uint64)]
    for r in range(3):
        for j in range(2):
            for x in keys:
                want = ((s[r][j] * oracle_mod.mix64(x)) & M64) >> (64 - L)
                assert o.pos(r, j, x) == want
                assert 0 <= want < m


@pytest.mark.parametrize("L", [1, 5, 20, 32])
def test_positions_uniform(oracle_mod, L):
    o = oracle_mod.Oracle(4, 2, 2, 1 << L, 2, 5)
    rng = np.random.default_rng(L)
    xs = rng.integers(0, 1 << 62, 20000, dtype=np.uint64)
    bins = 32 if L >= 5 else (1 << L)
    for r in range(2):
        for j in range(2):
            pos = np.array([o.pos(r, j, int(x)) for x in xs])
            assert pos.max() < (1 << L)
            h = np.bincount((pos * bins) >> L, minlength=bins)
            exp = xs.size / bins
            chi2 = ((h - exp) ** 2 / exp).sum()
            # chi-square with bins-1 dof; 99.99% quantile well under dof + 6*sqrt(2 dof)
            assert chi2 < (bins - 1) + 6 * np.sqrt(2 * (bins - 1)) + 5


def test_position_pairs_independent(oracle_mod):
    # different (r, j) multipliers give (nearly) independent positions: joint
    # occupancy of a 8x8 grid of position ranges is flat
    o = oracle_mod.Oracle(4, 2, 2, 1 << 20, 2, 11)
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 1 << 62, 20000, dtype=np.uint64)
    p0 = np.array([o.pos(0, 0, int(x)) for x in xs]) >> 17
    p1 = np.array([o.pos(1, 1, int(x)) for x in xs]) >> 17
    h = np.bincount(p0 * 8 + p1, minlength=64)
    exp = xs.size / 64
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 6 * np.sqrt(126) + 5


def test_kmer_closed_forms(oracle_mod):
    k = 31
    assert list(oracle_mod.kmers(b"A" * 31, k)) == [0]
    assert list(oracle_mod.kmers(b"T" * 31, k)) == [4**31 - 1]
    assert list(oracle_mod.kmers(b"C" + b"A" * 30, k)) == [4**30]
    assert list(oracle_mod.kmers(b"A" * 30 + b"G", k)) == [2]
    assert list(oracle_mod.kmers(b"ACGT", 4)) == [0 * 64 + 1 * 16 + 2 * 4 + 3]
    assert list(oracle_mod.kmers(b"acgt", 4)) == [27]
    assert list(oracle_mod.kmers(b"T" * 32, 32)) == [M64]
    # n - k + 1 windows; fewer than k bases -> none
    assert oracle_mod.kmers(b"A" * 40, k).size == 10
    assert oracle_mod.kmers(b"A" * 30, k).size == 0
    with pytest.raises(ValueError):
        oracle_mod.kmers(b"ACGTN" + b"A" * 30, k)
    with pytest.raises(ValueError):
        oracle_mod.kmers(b"A" * 31, 33)


def test_kmer_sliding_invariant(oracle_mod):
    rng = np.random.default_rng(4)
    seq = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 500)])
    code = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
    for k in (1, 7, 31, 32):
        ks = [int(v) for v in oracle_mod.kmers(seq, k)]
        mod = 4**k
        for p in range(len(ks) - 1):
            assert ks[p + 1] == (ks[p] * 4 + code[seq[p + k]]) % mod
        # the first window read as a base-4 numeral, most significant first
        assert ks[0] == int("".join(str(code[c]) for c in seq[:k]), 4)


CANON = 0x100


def _revcomp(seq: bytes) -> bytes:
    return bytes(seq[::-1]).translate(bytes.maketrans(b"ACGTacgt", b"TGCAtgca"))


def test_canonical_kmers_are_strand_independent(oracle_mod):
    # canonical key = min(window, reverse complement): a sequence and its
    # reverse complement give the same keys, in reverse order
    rng = np.random.default_rng(9)
    seq = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 400)])
    for k in (1, 2, 15, 31, 32):
        a = [int(v) for v in oracle_mod.kmers(seq, k | CANON)]
        b = [int(v) for v in oracle_mod.kmers(_revcomp(seq), k | CANON)]
        assert a == b[::-1]
        fwd = [int(v) for v in oracle_mod.kmers(seq, k)]
        rc = [int(v) for v in oracle_mod.kmers(_revcomp(seq), k)][::-1]
        assert a == [min(x, y) for x, y in zip(fwd, rc)]
    # closed forms (A=0 C=1 G=2 T=3): ACG -> min(ACG=6, CGT=27); TTT -> AAA = 0
    assert list(oracle_mod.kmers(b"ACG", 3 | CANON)) == [6]
    assert list(oracle_mod.kmers(b"TTT", 3 | CANON)) == [0]
    assert list(oracle_mod.kmers(b"GGG", 3 | CANON)) == [int("111", 4)]  # CCC
    with pytest.raises(ValueError):
        oracle_mod.kmers(b"ACGT", 3 | 0x400)  # no such flag (0x200 is skip-N)
