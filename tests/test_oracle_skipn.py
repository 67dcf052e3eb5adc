"""Pins for skip-N windows in the oracle (the sliding window of Sec. 3.2.1 over
reads that carry unresolved bases, as the k-mers of whole-genome reads in
Sec. 5.2 do).  Reading: with the SKIP_N flag in k, a window holding any byte
outside ACGTacgt is left out, and the sequence's terms are its other windows
in order; a query with no such window is a bad sequence.  Checked against
closed-form window counts, against keys computed here with Python integers
from the resolved runs, and against the oracle's own pinned key and Bloom
filter primitives (Algorithms 1 and 2)."""
import numpy as np
import pytest

SKIPN = 0x200
CANON = 0x100
CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3, ord("a"): 0, ord("c"): 1, ord("g"): 2, ord("t"): 3}
JUNK = b"NnRY-.\x00\xff"


def _key(s: bytes, k: int, canon: bool) -> int:
    fwd = 0
    for ch in s:
        fwd = fwd * 4 + CODE[ch]
    if not canon:
        return fwd
    rc = 0
    for ch in reversed(s):
        rc = rc * 4 + (3 - CODE[ch])
    return min(fwd, rc)


def _runs_keys(seq: bytes, k: int, canon: bool = False) -> list[int]:
    """Keys of the windows inside maximal runs of ACGTacgt, runs in order."""
    out, run = [], []
    for ch in seq + b"N":
        if ch in CODE:
            run.append(ch)
            continue
        r = bytes(run)
        out += [_key(r[p:p + k], k, canon) for p in range(len(r) - k + 1)]
        run = []
    return out


def _seq_with_junk(rng, n, p_junk):
    s = bytearray(rng.choice(list(b"ACGTacgt"), n).astype(np.uint8))
    for i in np.flatnonzero(rng.random(n) < p_junk):
        s[i] = JUNK[rng.integers(len(JUNK))]
    return bytes(s)


@pytest.mark.parametrize("n,k", [(50, 7), (80, 31), (40, 1), (64, 32)])
def test_single_unresolved_base_count_closed_form(oracle_mod, n, k):
    rng = np.random.default_rng(n + k)
    base = bytes(rng.choice(list(b"ACGT"), n).astype(np.uint8))
    for j in range(n):
        s = base[:j] + b"N" + base[j + 1:]
        want = max(0, j - k + 1) + max(0, n - j - 1 - k + 1)
        got = oracle_mod.kmers(s, k | SKIPN)
        assert got.size == want
        # without the flag the byte rejects the sequence
        with pytest.raises(ValueError):
            oracle_mod.kmers(s, k)


@pytest.mark.parametrize("k", [1, 5, 31, 32])
@pytest.mark.parametrize("canon", [False, True])
def test_keys_are_the_windows_of_the_resolved_runs(oracle_mod, k, canon):
    rng = np.random.default_rng(k * 3 + canon)
    flags = k | SKIPN | (CANON if canon else 0)
    for n, pj in [(200, 0.01), (200, 0.05), (120, 0.2), (40, 0.0), (300, 0.002)]:
        s = _seq_with_junk(rng, n, pj)
        got = [int(x) for x in oracle_mod.kmers(s, flags)]
        assert got == _runs_keys(s, k, canon)
    # no unresolved byte: the same keys as without the flag
    s = bytes(rng.choice(list(b"ACGTacgt"), 90).astype(np.uint8))
    assert np.array_equal(oracle_mod.kmers(s, flags), oracle_mod.kmers(s, flags & ~SKIPN))


def test_unresolved_bases_at_window_edges(oracle_mod):
    k = 31
    acgt = b"ACGT" * 8  # 32 bases
    assert oracle_mod.kmers(b"N" + acgt[:31], k | SKIPN).size == 1           # first byte
    assert oracle_mod.kmers(acgt[:31] + b"N", k | SKIPN).size == 1           # last byte
    assert oracle_mod.kmers(b"N" + acgt[:30] + b"N", k | SKIPN).size == 0    # both ends
    assert oracle_mod.kmers(acgt[:15] + b"N" + acgt[:15], k | SKIPN).size == 0  # middle of the only window
    assert oracle_mod.kmers(b"N" * 100, k | SKIPN).size == 0
    assert oracle_mod.kmers(b"", k | SKIPN).size == 0
    # the key of the window after the N is the plain key of those 31 bases
    assert int(oracle_mod.kmers(b"N" + acgt[:31], k | SKIPN)[0]) == _key(acgt[:31], 31, False)


def _pair(oracle_mod, K=12, B=4, R=3, m=1 << 14, eta=2, seed=9):
    return (oracle_mod.Oracle(K, B, R, m, eta, seed), oracle_mod.Oracle(K, B, R, m, eta, seed))


def test_insert_with_unresolved_bases_equals_inserting_the_valid_windows(oracle_mod):
    rng = np.random.default_rng(4)
    for canon in (False, True):
        flags = 31 | SKIPN | (CANON if canon else 0)
        a, b = _pair(oracle_mod)
        seqs = [_seq_with_junk(rng, int(rng.integers(20, 400)), pj) for pj in (0.0, 0.01, 0.03, 0.3, 1.0, 0.01)]
        ids = np.arange(len(seqs), dtype=np.uint64) * 2
        off = np.zeros(len(seqs) + 1, np.uint64)
        np.cumsum([len(x) for x in seqs], out=off[1:])
        a.insert_seq_batch(ids, np.frombuffer(b"".join(seqs), np.uint8), off, flags, nthreads=2)
        for i, s in zip(ids, seqs):
            b.insert_keys(int(i), np.array(_runs_keys(s, 31, canon), np.uint64))
        assert np.array_equal(a.cell_popcount(), b.cell_popcount())
        for r in range(a.R):
            for c in range(a.B):
                assert np.array_equal(a.export_bf(r, c), b.export_bf(r, c))
        assert np.array_equal(a.registered(), b.registered())  # sets with no window still register


def test_query_with_unresolved_bases_is_the_conjunction_of_its_valid_windows(oracle_mod):
    rng = np.random.default_rng(8)
    o = oracle_mod.Oracle(30, 6, 3, 1 << 16, 2, 3)
    sets = [bytes(rng.choice(list(b"ACGT"), 400).astype(np.uint8)) for _ in range(30)]
    for i, s in enumerate(sets):
        o.insert_seq(i, s, 31)
    queries, want = [], []
    for t in range(40):
        s = sets[int(rng.integers(30))]
        a = int(rng.integers(0, 300))
        q = bytearray(s[a:a + 100])
        for j in rng.integers(0, 100, int(rng.integers(0, 4))):
            q[j] = JUNK[int(rng.integers(len(JUNK)))]
        q = bytes(q)
        keys = _runs_keys(q, 31)
        if not keys:
            continue
        queries.append(q)
        want.append(o.query_keys(np.array(keys, np.uint64)))
        assert np.array_equal(o.query_seq(q, 31 | SKIPN), want[-1])
    off = np.zeros(len(queries) + 1, np.uint64)
    np.cumsum([len(x) for x in queries], out=off[1:])
    ids, ioff = o.query_batch("seq", np.frombuffer(b"".join(queries), np.uint8), off, k=31 | SKIPN, nthreads=2)
    for t, w in enumerate(want):
        assert np.array_equal(ids[int(ioff[t]):int(ioff[t + 1])], w)


def test_query_without_a_valid_window_is_a_bad_sequence(oracle_mod):
    from oracle.oracle import EBADSEQ, OracleError

    o = oracle_mod.Oracle(4, 2, 2, 1 << 10, 2, 1)
    o.insert_seq(0, b"ACGT" * 20, 31)
    for q in (b"N" * 40, b"ACGT" * 7 + b"N" + b"ACGT" * 7, b"ACG"):
        with pytest.raises(OracleError) as e:
            o.query_seq(q, 31 | SKIPN)
        assert e.value.code == EBADSEQ
    good = b"ACGT" * 8
    bad = b"N" * 40
    off = np.array([0, len(good), len(good) + len(bad)], np.uint64)
    with pytest.raises(OracleError) as e:
        o.query_batch("seq", np.frombuffer(good + bad, np.uint8), off, k=31 | SKIPN)
    assert e.value.code == EBADSEQ and "query 1" in str(e.value)
