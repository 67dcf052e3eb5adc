"""GPU parity: the CUDA library (called through the C ABI) against the CPU
oracle, element by element, on seeded synthetic workloads shaped like the
paper's (scaled so the oracle finishes in seconds, with several tiles and
ragged tails), plus edge cases.  Index bits, registered sets, the partition
table and every query's ID list must be identical."""
import numpy as np
import pytest

import synth
from tests.parity import assert_index_equal, assert_partition_equal, assert_query_equal, build_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from oracle.oracle import Oracle
    from paper_1910_02611_gb300 import Rambo

    return Rambo, Oracle


def _w(name, scale, **kw):
    return synth.make(name, scale, **kw)


WORKLOADS = {
    "tiny_full": lambda: _w("tiny", 1.0),
    "genome_small": lambda: _w("genome", 0.02, m=1 << 18),
    "uneven_small": lambda: _w("uneven", 0.004, m=1 << 16, n_queries=750_000),  # 3000 queries at this scale
    "document_small": lambda: _w("document", 0.01, m=1 << 16),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def pair(request, mods):
    Rambo, Oracle = mods
    w = WORKLOADS[request.param]()
    g, o = build_pair(w, Rambo, Oracle, insert_chunks=3)
    yield w, g, o
    g.close()


def test_index_bits_identical(pair):
    w, g, o = pair
    assert_index_equal(g, o)
    assert_partition_equal(g, o)


def test_cell_popcount_identical(pair):
    w, g, o = pair
    assert np.array_equal(g.cell_popcount(), o.cell_popcount())


def test_queries_identical_default_config(pair):
    w, g, o = pair
    assert_query_equal(g, o, w.queries, k=w.k)
    st = g.last_query_stats()
    assert st["keys_probed"] <= st["keys_submitted"]
    assert st["keys_probed"] * w.eta <= st["rows_read"] <= st["keys_probed"] * w.R * w.eta


def test_queries_identical_every_kernel_config(pair):
    w, g, o = pair
    base = g.get_config()
    q = w.queries.subset(np.arange(min(len(w.queries), 800)))
    try:
        for cfg in g.list_configs():
            for stage in (1, 2, 3):
                for order in (0, 1, 2):
                    g.set_config(**{**cfg, "set_stage": stage, "visit_order": order})
                    assert_query_equal(g, o, q, k=w.k)
        # queries shared by 2, 4 or 8 warps of a block, forced, then chosen
        # from the batch size (small batches take whole blocks per query)
        for wpq in (1, 2, 4, 8):
            for stage in (0, 1, 2, 3):
                g.set_config(**{**base, "warps_per_query": wpq, "set_stage": stage})
                assert_query_equal(g, o, q, k=w.k)
        g.set_config(**base)
        for n in (1, 3, 37):
            assert_query_equal(g, o, w.queries.subset(np.arange(min(n, len(w.queries)))), k=w.k)
        g.set_config(**{**base, "l2_fetch_bytes": 32})
        assert_query_equal(g, o, q, k=w.k)
        g.set_config(**{**base, "cluster": 1})
        assert_query_equal(g, o, w.queries, k=w.k)
        for load in range(8):  # every cache operator / L2 prefetch-size hint of the row reads
            g.set_config(**{**base, "row_load": load})
            assert_query_equal(g, o, q, k=w.k)
    finally:
        g.set_config(**base)


def test_device_inputs_match_host_inputs(pair):
    import torch

    w, g, o = pair
    q = w.queries.subset(np.arange(min(len(w.queries), 500)))
    hid, hoff = g.query(q.data, q.offsets, kind=q.kind, k=w.k)
    dt = torch.from_numpy(q.data.view(np.int64) if q.kind == "keys" else q.data).cuda()
    do = torch.from_numpy(q.offsets.view(np.int64)).cuda()
    did, doff = g.query(dt, do, kind=q.kind, k=w.k)
    assert np.array_equal(hoff, doff.cpu().numpy().view(np.uint64))
    assert np.array_equal(hid, did.cpu().numpy().view(np.uint32))


def test_query_into_and_nospc(pair):
    from paper_1910_02611_gb300 import ENOSPC, RamboError

    w, g, o = pair
    q = w.queries.subset(np.arange(min(len(w.queries), 300)))
    ids, off = g.query(q.data, q.offsets, kind=q.kind, k=w.k)
    n = len(q)
    out_ids = np.zeros(ids.size + 5, np.uint32)
    out_off = np.zeros(n + 1, np.uint64)
    got = g.query_into(q.data, q.offsets, out_ids, out_off, kind=q.kind, k=w.k)
    assert got == ids.size
    assert np.array_equal(out_off, off) and np.array_equal(out_ids[:got], ids)
    if ids.size:
        with pytest.raises(RamboError) as e:
            g.query_into(q.data, q.offsets, np.zeros(ids.size - 1, np.uint32), out_off, kind=q.kind, k=w.k)
        assert e.value.code == ENOSPC


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def _rand_seq(rng, n):
    return np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)]


@pytest.mark.parametrize("B,R,m,eta", [(1, 1, 1 << 10, 1), (33, 2, 2, 3), (100, 8, 1 << 12, 4), (320, 5, 1 << 11, 2),
                                       (4096, 1, 1 << 8, 2), (7, 8, 1 << 14, 3)])
def test_edge_parameters(mods, B, R, m, eta):
    Rambo, Oracle = mods
    rng = np.random.default_rng(B * 1000 + R)
    K = 37  # not a multiple of 32
    lens = rng.integers(0, 400, K)
    lens[3] = 0   # empty set
    lens[5] = 30  # shorter than k: registered, no k-mers
    seqs = [_rand_seq(rng, int(n)) for n in lens]
    bases = np.concatenate(seqs)
    off = np.zeros(K + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    ids = rng.permutation(np.arange(K, dtype=np.uint64))  # sets inserted in shuffled ID order
    perm_seqs = [seqs[int(i)] for i in ids]
    pb = np.concatenate(perm_seqs)
    poff = np.zeros(K + 1, np.uint64)
    np.cumsum([s.size for s in perm_seqs], out=poff[1:])
    g = Rambo(K + 3, B, R, m, eta, 7)  # capacity beyond the inserted IDs
    o = Oracle(K + 3, B, R, m, eta, 7)
    g.insert(ids, pb, poff, kind="seq", k=31)
    o.insert_seq_batch(ids, pb, poff, 31)
    assert_index_equal(g, o)
    # queries: substrings of exactly k bases, long ones, lower case, fresh random
    qs = []
    for t in range(120):
        i = int(rng.integers(0, K))
        s = seqs[i]
        if s.size >= 31 and t % 4:
            a = int(rng.integers(0, s.size - 30))
            b = int(rng.integers(a + 31, min(s.size, a + 200) + 1))
            q = s[a:b].copy()
        else:
            q = _rand_seq(rng, int(rng.integers(31, 90)))
        if t % 7 == 0:
            q = np.frombuffer(bytes(q).lower(), np.uint8)
        qs.append(q)
    qd = np.concatenate(qs)
    qo = np.zeros(len(qs) + 1, np.uint64)
    np.cumsum([q.size for q in qs], out=qo[1:])
    assert_query_equal(g, o, synth.Collection("seq", qd, qo), k=31)
    # key queries of 1..6 keys, some repeated
    keys = rng.integers(0, 1 << 62, 300, dtype=np.uint64)
    g2 = Rambo(K, B, R, m, eta, 9)
    o2 = Oracle(K, B, R, m, eta, 9)
    koff = np.linspace(0, keys.size, K + 1).astype(np.uint64)
    g2.insert(np.arange(K, dtype=np.uint64), keys, koff)
    o2.insert_keys_batch(np.arange(K, dtype=np.uint64), keys, koff)
    assert_index_equal(g2, o2)
    ql = [np.concatenate([rng.choice(keys, int(rng.integers(1, 6))), rng.choice(keys, int(rng.integers(0, 2)))])
          for _ in range(200)]
    ql += [rng.integers(0, 1 << 62, 1, dtype=np.uint64) for _ in range(50)]
    qk = np.concatenate(ql).astype(np.uint64)
    qko = np.zeros(len(ql) + 1, np.uint64)
    np.cumsum([q.size for q in ql], out=qko[1:])
    assert_query_equal(g2, o2, synth.Collection("keys", qk, qko))


def test_kmer_lengths_other_than_31(mods):
    Rambo, Oracle = mods
    rng = np.random.default_rng(5)
    for k in (1, 5, 16, 32):
        K, B, R, m, eta = 12, 9, 3, 1 << 12, 2
        lens = rng.integers(k, 300, K)
        bases = _rand_seq(rng, int(lens.sum()))
        off = np.zeros(K + 1, np.uint64)
        np.cumsum(lens, out=off[1:])
        g = Rambo(K, B, R, m, eta, k)
        o = Oracle(K, B, R, m, eta, k)
        g.insert(np.arange(K, dtype=np.uint64), bases, off, kind="seq", k=k)
        o.insert_seq_batch(np.arange(K, dtype=np.uint64), bases, off, k)
        assert_index_equal(g, o)
        n_q = int(bases.size // 60)
        qo = np.arange(0, n_q * 60 + 1, 60, dtype=np.uint64)
        qd = bases[: int(qo[-1])]
        assert_query_equal(g, o, synth.Collection("seq", qd.copy(), qo), k=k)


def test_offsets_not_starting_at_zero_and_empty_batch(mods):
    Rambo, Oracle = mods
    rng = np.random.default_rng(6)
    K = 20
    keys = rng.integers(0, 1 << 62, 1000, dtype=np.uint64)
    g = Rambo(K, 16, 3, 1 << 12, 2, 3)
    o = Oracle(K, 16, 3, 1 << 12, 2, 3)
    off = np.linspace(100, 900, K + 1).astype(np.uint64)  # uses keys[100:900]
    g.insert(np.arange(K, dtype=np.uint64), keys, off)
    o.insert_keys_batch(np.arange(K, dtype=np.uint64), keys, off)
    assert_index_equal(g, o)
    qo = np.arange(50, 251, 2, dtype=np.uint64)
    assert_query_equal(g, o, synth.Collection("keys", keys, qo))
    ids, offs = g.query(keys, np.array([7], np.uint64))  # no queries
    assert ids.size == 0 and list(offs) == [0]
    g.insert(np.zeros(0, np.uint64), keys, np.array([0], np.uint64))  # no sets: nothing happens
    assert_index_equal(g, o)


def test_errors_leave_the_index_unchanged(mods):
    from paper_1910_02611_gb300 import EBADSEQ, EINVAL, ERANGE, RamboError

    Rambo, Oracle = mods
    rng = np.random.default_rng(8)
    K = 10
    g = Rambo(K, 8, 2, 1 << 10, 2, 1)
    o = Oracle(K, 8, 2, 1 << 10, 2, 1)
    seqs = _rand_seq(rng, 500)
    off = np.array([0, 100, 250, 500], np.uint64)
    g.insert(np.array([1, 2, 3], np.uint64), seqs, off, kind="seq")
    o.insert_seq_batch(np.array([1, 2, 3], np.uint64), seqs, off, 31)
    before = g.export_index().copy()

    def expect(code, item, fn):
        with pytest.raises(RamboError) as e:
            fn()
        assert e.value.code == code
        if item is not None:
            assert e.value.item == item

    bad = seqs.copy()
    bad[260] = ord("N")
    expect(EBADSEQ, 2, lambda: g.insert(np.array([4, 5, 6], np.uint64), bad, off, kind="seq"))
    expect(ERANGE, 1, lambda: g.insert(np.array([4, 10, 6], np.uint64), seqs, off, kind="seq"))
    expect(EINVAL, 1, lambda: g.insert(np.array([4, 5, 6], np.uint64), seqs, np.array([0, 300, 250, 500], np.uint64),
                                       kind="seq"))
    assert np.array_equal(before, g.export_index())
    assert not g.export_registered()[4]
    # queries
    qoff = np.array([0, 40, 100, 131], np.uint64)
    expect(EBADSEQ, 1, lambda: g.query(bad[220:351], qoff, kind="seq"))  # bad base at 260-220=40 -> query 1
    expect(EBADSEQ, 2, lambda: g.query(seqs, np.array([0, 40, 100, 120], np.uint64), kind="seq"))  # 20 < k
    expect(EINVAL, 1, lambda: g.query(rng.integers(0, 9, 10, dtype=np.uint64), np.array([0, 3, 3, 10], np.uint64)))
    expect(EINVAL, None, lambda: g.query(rng.integers(0, 9, 10, dtype=np.uint64), np.array([0, 5, 3, 10], np.uint64)))
    # a good query afterwards still works
    q = synth.Collection("seq", seqs[:200].copy(), np.array([0, 60, 200], np.uint64))
    assert_query_equal(g, o, q)


def test_duplicate_and_repeated_inserts(mods):
    Rambo, Oracle = mods
    rng = np.random.default_rng(9)
    K = 40
    keys = rng.integers(0, 1 << 62, 2000, dtype=np.uint64)
    off = np.linspace(0, 2000, 21).astype(np.uint64)
    ids = rng.integers(0, K, 20).astype(np.uint64)  # repeated IDs
    g = Rambo(K, 12, 4, 1 << 13, 3, 5)
    o = Oracle(K, 12, 4, 1 << 13, 3, 5)
    for _ in range(2):  # inserting twice changes nothing
        g.insert(ids, keys, off)
    o.insert_keys_batch(ids, keys, off)
    assert_index_equal(g, o)


def test_save_load_roundtrip(mods, tmp_path):
    Rambo, Oracle = mods
    w = synth.make("genome", 0.01, m=1 << 14)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    p = str(tmp_path / "idx.rambo")
    g.save(p)
    h = Rambo.load(p)
    assert np.array_equal(g.export_index(), h.export_index())
    assert np.array_equal(g.export_registered(), h.export_registered())
    a = g.query(w.queries.data, w.queries.offsets, kind="seq")
    b = h.query(w.queries.data, w.queries.offsets, kind="seq")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("tile_bytes", [1 << 20, 3 << 20])
def test_tiled_construction_matches_oracle(mods, tile_bytes):
    # the build forced to run window by window over the index (L2-sized
    # windows in production; small ones here so many tiles and a ragged last
    # tile are exercised)
    Rambo, Oracle = mods
    w = synth.make("genome", 0.02, m=1 << 18)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.set_build_tiling(tile_bytes, mode=1)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31, nthreads=8)
    assert_index_equal(g, o)
    assert_query_equal(g, o, w.queries.subset(np.arange(1000)))
    # keys input, forced untiled, same bits
    keys = np.random.default_rng(3).integers(0, 1 << 62, 50000, dtype=np.uint64)
    off = np.linspace(0, keys.size, 11).astype(np.uint64)
    for mode in (1, 2):
        g2 = Rambo(10, 40, 3, 1 << 17, 2, 5)
        g2.set_build_tiling(tile_bytes, mode=mode)
        g2.insert(np.arange(10, dtype=np.uint64), keys, off)
        o2 = Oracle(10, 40, 3, 1 << 17, 2, 5)
        o2.insert_keys_batch(np.arange(10, dtype=np.uint64), keys, off)
        assert_index_equal(g2, o2)


@pytest.mark.parametrize("name,k", [("genome_small", 31), ("genome_small", 31 | 0x100), ("document_small", 31),
                                    ("uneven_small", 31 | 0x200)])
def test_bucketed_construction_matches_oracle(mods, name, k):
    # construction mode 3: every key hashed once per input chunk, its updates
    # filed by window of the index and applied window by window -- the same
    # bits as the oracle's Algorithm 1 and as the window-by-window build
    Rambo, Oracle = mods
    w = WORKLOADS[name]()
    kind = w.sets.kind
    g = Rambo(w.K, w.B, w.R, 1 << 22, w.eta, w.seed)  # an index of several 48 MiB windows
    g.set_build_tiling(mode=3)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind=kind, k=k)
    o = Oracle(w.K, w.B, w.R, 1 << 22, w.eta, w.seed)
    if kind == "keys":
        o.insert_keys_batch(w.sets.ids, w.sets.data, w.sets.offsets, nthreads=8)
    else:
        o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, k, nthreads=8)
    assert np.array_equal(g.cell_popcount(), o.cell_popcount())
    gt = Rambo(w.K, w.B, w.R, 1 << 22, w.eta, w.seed)
    gt.set_build_tiling(1 << 24, mode=1)
    gt.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind=kind, k=k)
    assert np.array_equal(gt.export_index(), g.export_index())
    rows = g.export_index()
    for r in range(w.R):  # sampled rows against the oracle's row view
        for p in np.random.default_rng(r).integers(0, 1 << 22, 300):
            want = o.get_row(r, int(p)).view(np.uint32)[: g.row_words]
            assert np.array_equal(rows[r, int(p), : g.row_words], want)
    gt.close()
    g.close()


def test_bucketed_construction_recovers_from_skewed_keys(mods):
    # one key repeated 300000 times lands every update of the batch in the few
    # rows it hashes to: a bucket overflows and the chunk is filed again
    Rambo, Oracle = mods
    K, B, R, m, eta = 40, 64, 6, 1 << 22, 2
    keys = np.full(300_000, 0x1234567, np.uint64)
    keys[::1000] = np.arange(300, dtype=np.uint64) * 7919  # and a few others
    off = np.array([0, 150_000, 300_000], np.uint64)
    ids = np.array([3, 17], np.uint64)
    g = Rambo(K, B, R, m, eta, 42)
    g.set_build_tiling(mode=3)
    g.insert(ids, keys, off, kind="keys")
    o = Oracle(K, B, R, m, eta, 42)
    o.insert_keys_batch(ids, keys, off)
    assert np.array_equal(g.cell_popcount(), o.cell_popcount())
    assert_index_equal(g, o)
    g.close()


def test_pack_aligned_and_unaligned_inputs(mods):
    # sequences starting at every alignment of the base array (16-byte vector
    # path and byte path of the packer), with and without a bad byte
    import torch

    from paper_1910_02611_gb300 import EBADSEQ, RamboError

    Rambo, Oracle = mods
    rng = np.random.default_rng(21)
    seqs = _rand_seq(rng, 3000)
    g = Rambo(8, 16, 3, 1 << 12, 2, 4)
    o = Oracle(8, 16, 3, 1 << 12, 2, 4)
    off = np.array([0, 400, 900, 1500, 2100, 2500, 2800, 2900, 3000], np.uint64)
    g.insert(np.arange(8, dtype=np.uint64), seqs, off, kind="seq")
    o.insert_seq_batch(np.arange(8, dtype=np.uint64), seqs, off, 31)
    dev_bases = torch.from_numpy(seqs.copy()).cuda()
    for start in (0, 1, 3, 8, 13, 16, 31):
        qo = np.arange(start, start + 20 * 97 + 1, 97, dtype=np.uint64)
        ids, offs = g.query(dev_bases, torch.from_numpy(qo.view(np.int64)).cuda(), kind="seq")
        rids, roff = o.query_batch("seq", seqs, qo, k=31)
        assert np.array_equal(offs.cpu().numpy().view(np.uint64), roff)
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), rids)
        for bad_at in (start + 5, start + 97 * 3 + 31, start + 97 * 7):
            b = seqs.copy()
            b[bad_at] = ord("x")
            with pytest.raises(RamboError) as e:
                g.query(torch.from_numpy(b).cuda(), torch.from_numpy(qo.view(np.int64)).cuda(), kind="seq")
            assert e.value.code == EBADSEQ and e.value.item == (bad_at - start) // 97


def test_one_query_per_launch_baseline_matches_oracle(mods):
    import torch

    Rambo, Oracle = mods
    for name, kw in (("genome", dict(m=1 << 18)), ("document", dict(m=1 << 16))):
        w = synth.make(name, 0.01, **kw)
        g, o = build_pair(w, Rambo, Oracle)
        q = w.queries.subset(np.arange(min(300, len(w.queries))))
        dd = torch.from_numpy(q.data.view(np.int64) if q.kind == "keys" else q.data).cuda()
        ids, off = g.query_one_per_launch(dd, q.offsets, kind=q.kind, k=w.k)
        rids, roff = o.query_batch(q.kind, q.data, q.offsets, k=w.k)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)


def test_autotune_picks_a_config_and_results_stay_identical(mods):
    Rambo, Oracle = mods
    w = synth.make("genome", 0.02, m=1 << 18)
    g, o = build_pair(w, Rambo, Oracle)
    q = w.queries.subset(np.arange(500))
    best = g.autotune(q.data, q.offsets, kind="seq", reps=2)
    assert best == g.get_config()
    assert best["visit_order"] in (1, 2)
    assert_query_equal(g, o, w.queries)


@pytest.mark.parametrize("B,folds", [(64, 1), (640, 3), (320, 2), (10, 1)])
def test_folding_over_equals_an_index_built_with_half_the_cells(mods, B, folds):
    # appendix "folding over": OR of cell b + B/2 onto cell b.  With the same
    # seed the folded index equals the oracle (and a GPU index) built with
    # B / 2^folds cells from the same sets.
    Rambo, Oracle = mods
    w = synth.make("genome", 0.01, m=1 << 15, B=B, R=4)
    g = Rambo(w.K, B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    for _ in range(folds):
        g.fold()
    B2 = B >> folds
    o = Oracle(w.K, B2, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31)
    assert g.B == B2
    assert_index_equal(g, o)
    assert_partition_equal(g, o)
    assert_query_equal(g, o, w.queries)
    direct = Rambo(w.K, B2, w.R, w.m, w.eta, w.seed)
    direct.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    assert np.array_equal(direct.export_index(), g.export_index())


def test_large_host_batches_take_the_copy_pipeline(mods):
    # batches of 65536+ queries answered into host memory run in chunks whose
    # answers are copied while later chunks compute; the first call of a size
    # sizes the buffers the unpipelined way, the next ones pipeline.  Answers,
    # and the item an error is reported at, must not depend on the path.
    from paper_1910_02611_gb300 import EBADSEQ, EINVAL, RamboError

    Rambo, Oracle = mods
    w = synth.make("genome", 0.02, m=1 << 18)
    g, o = build_pair(w, Rambo, Oracle)
    rng = np.random.default_rng(64)
    for n in (70_000, 70_000, 600_000):
        q = synth.substring_queries(rng, w.sets, rng.integers(31, 60, n))
        ids, off = g.query(q.data, q.offsets, kind="seq")
        if n == 600_000:  # the oracle checks a sample; the rest against the device-output path
            import torch

            dids, doff = g.query(torch.from_numpy(q.data).cuda(), torch.from_numpy(q.offsets.view(np.int64)).cuda(),
                                 kind="seq")
            assert np.array_equal(off, doff.cpu().numpy().view(np.uint64))
            assert np.array_equal(ids, dids.cpu().numpy().view(np.uint32))
            sel = np.sort(rng.choice(n, 3000, replace=False))
            sub = q.subset(sel)
            rids, roff = o.query_batch("seq", sub.data, sub.offsets, k=31)
            for j, t in enumerate(sel):
                assert np.array_equal(ids[int(off[t]):int(off[t + 1])], rids[int(roff[j]):int(roff[j + 1])])
        else:
            rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
            assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    # errors in a late chunk: the item index is the batch's, not the chunk's
    q = synth.substring_queries(rng, w.sets, rng.integers(31, 60, 70_000))
    bad = q.data.copy()
    bad[int(q.offsets[65_000]) + 3] = ord("N")
    with pytest.raises(RamboError) as e:
        g.query(bad, q.offsets, kind="seq")
    assert e.value.code == EBADSEQ and e.value.item == 65_000
    off = q.offsets.copy()
    off[50_001] = off[50_000] - 1  # query 50000 ends before it starts
    with pytest.raises(RamboError) as e:
        g.query(q.data, off, kind="seq")
    assert e.value.code == EINVAL and e.value.item == 50_000
    ids, off2 = g.query(q.data, q.offsets, kind="seq")  # and the handle still answers
    rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
    assert np.array_equal(off2, roff) and np.array_equal(ids, rids)
    g.close()


def test_fold_is_refused_while_a_plan_holds_the_index(mods):
    # A plan's captured graph reads the handle's rows and set-stage tables;
    # folding replaces them, so it must be refused (RAMBO_ESTATE, index
    # untouched) while the plan lives, and allowed once it is gone.
    from paper_1910_02611_gb300 import ESTATE, Plan, RamboError

    Rambo, Oracle = mods
    w = synth.make("genome", 0.01, m=1 << 15, B=64, R=4)
    g = Rambo(w.K, 64, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    before = g.export_index()
    q = w.queries.subset(np.arange(50))
    plan = Plan(g, "seq", max_queries=64, max_items=int(q.offsets[-1]) + 64, max_ids=1 << 16)
    plan.launch_host(q.data, q.offsets)
    ids_a, off_a = plan.wait()
    with pytest.raises(RamboError) as e:
        g.fold()
    assert e.value.code == ESTATE
    assert g.B == 64 and np.array_equal(g.export_index(), before)
    # the plan still answers as before
    plan.launch_host(q.data, q.offsets)
    ids_b, off_b = plan.wait()
    assert np.array_equal(ids_a, ids_b) and np.array_equal(off_a, off_b)
    plan.close()
    g.fold()
    assert g.B == 32
    o = Oracle(w.K, 32, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31)
    assert_index_equal(g, o)
    g.close()


def test_single_set_insert_host_and_device(mods):
    import torch

    Rambo, Oracle = mods
    rng = np.random.default_rng(40)
    K = 25
    g = Rambo(K, 20, 3, 1 << 12, 2, 8)
    o = Oracle(K, 20, 3, 1 << 12, 2, 8)
    for i in range(K):
        keys = rng.integers(0, 1 << 62, int(rng.integers(0, 300)), dtype=np.uint64)
        if i % 2:
            g.insert_set(i, keys)
        else:
            g.insert_set(i, torch.from_numpy(keys.view(np.int64)).cuda())
        o.insert_keys(i, keys)
    assert_index_equal(g, o)


@pytest.mark.parametrize("k", [31, 32, 7])
def test_canonical_kmers_index_and_queries(mods, k):
    Rambo, Oracle = mods
    CANON = 0x100
    w = synth.make("genome", 0.01, m=1 << 16)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq", k=k | CANON)
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, k | CANON)
    assert_index_equal(g, o)
    # window-by-window build (keys hashed once, then streamed per window): same bits
    gt = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    gt.set_build_tiling(1 << 17, mode=1)
    gt.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq", k=k | CANON)
    assert np.array_equal(gt.export_index(), g.export_index())
    gt.close()
    q = w.queries.subset(np.arange(400))
    assert_query_equal(g, o, q, k=k | CANON)
    # the reverse-complemented queries give the same answers
    tr = bytes.maketrans(b"ACGT", b"TGCA")
    rc = [np.frombuffer(bytes(q.item(t)[::-1]).translate(tr), np.uint8) for t in range(len(q))]
    rq = synth.Collection("seq", np.concatenate(rc), q.offsets - q.offsets[0])
    a_ids, a_off = g.query(q.data, q.offsets, kind="seq", k=k | CANON)
    b_ids, b_off = g.query(rq.data, rq.offsets, kind="seq", k=k | CANON)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_off, b_off)
    # plain one-query-per-launch kernel agrees as well
    import torch

    ids1, off1 = g.query_one_per_launch(torch.from_numpy(q.data).cuda(), q.offsets, kind="seq", k=k | CANON)
    assert np.array_equal(ids1, a_ids) and np.array_equal(off1, a_off)


def _sprinkle_unresolved(rng, data: np.ndarray, rate: float, runs: int) -> np.ndarray:
    """A copy of ASCII DNA with single unresolved bytes at the given rate
    plus a few runs of N (as assembly gaps and low-quality stretches give)."""
    out = data.copy()
    junk = np.frombuffer(b"NnRY-.", np.uint8)
    hit = np.flatnonzero(rng.random(out.size) < rate)
    out[hit] = junk[rng.integers(0, junk.size, hit.size)]
    for _ in range(runs):
        a = int(rng.integers(0, max(1, out.size - 200)))
        out[a: a + int(rng.integers(1, 200))] = ord("N")
    return out


@pytest.mark.parametrize("k", [31, 31 | 0x100, 12])
def test_skip_n_windows_index_and_queries(mods, k):
    # skip-N (Sec. 3.2.1 over reads with unresolved bases): windows holding a
    # byte outside ACGTacgt are left out on both sides
    from paper_1910_02611_gb300 import EBADSEQ, Plan, RamboError

    Rambo, Oracle = mods
    SKIPN = 0x200
    rng = np.random.default_rng(k)
    w = synth.make("genome", 0.01, m=1 << 16)
    sets = synth.Collection("seq", _sprinkle_unresolved(rng, w.sets.data, 0.002, 40), w.sets.offsets, w.sets.ids)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(sets.ids, sets.data, sets.offsets, kind="seq", k=k | SKIPN)
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(sets.ids, sets.data, sets.offsets, k | SKIPN, nthreads=4)
    assert_index_equal(g, o)
    gt = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)  # window-by-window build
    gt.set_build_tiling(1 << 17, mode=1)
    gt.insert(sets.ids, sets.data, sets.offsets, kind="seq", k=k | SKIPN)
    assert np.array_equal(gt.export_index(), g.export_index())
    gt.close()
    # queries with unresolved bytes, some at the window edges; keep those with a valid window
    q = w.queries.subset(np.arange(600))
    qd = _sprinkle_unresolved(rng, q.data, 0.004, 3)
    for t in range(0, 600, 7):
        qd[int(q.offsets[t])] = ord("N")
        qd[int(q.offsets[t + 1]) - 1] = ord("n")
    keep = [t for t in range(600) if o.kmers_count(qd[int(q.offsets[t]):int(q.offsets[t + 1])], k | SKIPN) > 0]
    qq = synth.Collection("seq", qd, q.offsets).subset(np.array(keep))
    for cfg in ({}, {"set_stage": 1}, {"set_stage": 2}, {"set_stage": 3}, {"visit_order": 0}):
        if cfg:
            g.set_config(**cfg)
        assert_query_equal(g, o, qq, k=k | SKIPN)
    rids, roff = o.query_batch("seq", qq.data, qq.offsets, k=k | SKIPN)
    # through a captured plan
    plan = Plan(g, "seq", max_queries=len(qq), max_items=int(qq.offsets[-1]), max_ids=1 << 20, k=k | SKIPN)
    plan.launch_host(qq.data, qq.offsets)
    pids, poff = plan.wait()
    assert np.array_equal(poff, roff) and np.array_equal(pids, rids)
    plan.close()
    # the one-query-per-launch kernel
    import torch

    sub = qq.subset(np.arange(50))
    bids, boff = g.query_one_per_launch(torch.from_numpy(sub.data).cuda(), sub.offsets, kind="seq", k=k | SKIPN)
    s_ids, s_off = o.query_batch("seq", sub.data, sub.offsets, k=k | SKIPN)
    assert np.array_equal(boff, s_off) and np.array_equal(bids, s_ids)
    # a query with no valid window is a bad sequence, reported at its index
    bad = qq.subset(np.arange(10))
    bd = bad.data.copy()
    bd[int(bad.offsets[6]): int(bad.offsets[7])] = ord("N")
    with pytest.raises(RamboError) as e:
        g.query(bd, bad.offsets, kind="seq", k=k | SKIPN)
    assert e.value.code == EBADSEQ and e.value.item == 6
    # without the flag the same bytes reject the sequence
    with pytest.raises(RamboError) as e:
        g.query(qq.data, qq.offsets, kind="seq", k=k)
    assert e.value.code == EBADSEQ
    g.close()


def test_two_level_hash_node_indexes_merge_into_the_stacked_index(mods, tmp_path):
    # Sec. 5.2 / appendix: node-local builds (each inserting only the sets tau
    # routes to it) OR into the stacked index; it equals the oracle's stacked
    # structure, also after folding over and after a save/load round trip.
    Rambo, Oracle = mods
    w = synth.make("genome", 0.02, m=1 << 15)
    Bl, nodes = 16, 4
    whole = Rambo.stacked(w.K, Bl, nodes, w.R, w.m, w.eta, w.seed, tau_seed=12)
    whole.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    o = Oracle(w.K, Bl, w.R, w.m, w.eta, w.seed, nodes=nodes, tau_seed=12)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31)
    assert_index_equal(whole, o)
    assert_partition_equal(whole, o)
    assert [whole.node_of(i) for i in range(w.K)] == [o.node(i) for i in range(w.K)]
    parts = []
    for t in range(nodes):
        sel = np.array([i for i in range(len(w.sets)) if whole.node_of(int(w.sets.ids[i])) == t])
        g = Rambo.stacked(w.K, Bl, nodes, w.R, w.m, w.eta, w.seed, tau_seed=12)
        if sel.size:
            sub = w.sets.subset(sel)
            g.insert(sub.ids, sub.data, sub.offsets, kind="seq")
        parts.append(g)
    for g in parts[1:]:
        parts[0].merge(g)
    assert np.array_equal(parts[0].export_index(), whole.export_index())
    assert np.array_equal(parts[0].export_registered(), whole.export_registered())
    assert_query_equal(parts[0], o, w.queries)
    # folding over the stacked index
    parts[0].fold()
    o.fold()
    assert_index_equal(parts[0], o)
    assert_partition_equal(parts[0], o)
    assert_query_equal(parts[0], o, w.queries)
    p = str(tmp_path / "stacked.rambo")
    parts[0].save(p)
    back = Rambo.load(p)
    assert np.array_equal(back.export_index(), parts[0].export_index())
    assert_query_equal(back, o, w.queries.subset(np.arange(300)))
    # mismatched parameters do not merge
    from paper_1910_02611_gb300 import EINVAL, RamboError

    other = Rambo.stacked(w.K, Bl, nodes, w.R, w.m, w.eta, w.seed, tau_seed=13)
    with pytest.raises(RamboError) as e:
        whole.merge(other)
    assert e.value.code == EINVAL


def test_set_stages_follow_registration_across_inserts_merge_and_load(mods, tmp_path):
    # Algorithm 2 reports only inserted sets (registered IDs).  The sparse
    # stage enumerates registered members of the hit cells, so its tables must
    # follow every change of registration: later inserts of new IDs (also
    # seen by a plan captured before them), a merge, and a load.
    Rambo, Oracle = mods
    from paper_1910_02611_gb300 import Plan

    w = synth.make("document", 0.01, m=1 << 16)
    n = len(w.sets)
    halves = [w.sets.subset(np.arange(0, n // 2)), w.sets.subset(np.arange(n // 2, n))]
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    q = w.queries.subset(np.arange(400))
    base = g.get_config()
    plan = Plan(g, "keys", len(q), int(q.offsets[-1]), 1 << 22)

    def check_all(index):
        try:
            for stage in (0, 1, 2, 3):
                index.set_config(**{**base, "set_stage": stage})
                assert_query_equal(index, o, q)
        finally:
            index.set_config(**base)

    for part in halves:
        g.insert(part.ids, part.data, part.offsets, kind="keys")
        o.insert_keys_batch(part.ids, part.data, part.offsets)
        check_all(g)
        plan.launch_host(q.data, q.offsets)
        ids, off = plan.wait()
        rids, roff = o.query_batch("keys", q.data, q.offsets)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    # two indexes over the two halves, merged
    a = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    b = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    a.insert(halves[0].ids, halves[0].data, halves[0].offsets, kind="keys")
    b.insert(halves[1].ids, halves[1].data, halves[1].offsets, kind="keys")
    a.merge(b)
    check_all(a)
    p = str(tmp_path / "doc.rambo")
    a.save(p)
    check_all(Rambo.load(p))


def test_pinned_host_bases_read_in_place(mods):
    # Sequence batches in pinned host memory (>= 1 MiB) are packed straight
    # from host memory; results equal the oracle and the pageable-input path.
    import torch

    Rambo, Oracle = mods
    w = synth.make("genome", 0.02, m=1 << 18)
    g, o = build_pair(w, Rambo, Oracle)
    reps = 1 + (3 << 20) // max(1, int(w.queries.offsets[-1]))
    q = w.queries.subset(np.tile(np.arange(len(w.queries)), reps))
    assert int(q.offsets[-1]) >= (1 << 20)
    pinned = torch.from_numpy(q.data).pin_memory().numpy()
    ids_p, off_p = g.query(pinned, q.offsets, kind="seq")
    ids_h, off_h = g.query(q.data.copy(), q.offsets, kind="seq")
    rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
    assert np.array_equal(off_p, roff) and np.array_equal(ids_p, rids)
    assert np.array_equal(off_h, roff) and np.array_equal(ids_h, rids)
    # a bad base in pinned memory is reported like any other
    bad = pinned.copy()
    pinned2 = torch.from_numpy(bad).pin_memory().numpy()
    at = int(q.offsets[5]) + 3
    pinned2[at] = ord("N")
    from paper_1910_02611_gb300 import EBADSEQ, RamboError

    with pytest.raises(RamboError) as e:
        g.query(pinned2, q.offsets, kind="seq")
    assert e.value.code == EBADSEQ
    g.close()


def test_large_answers_into_pinned_and_pageable_host_buffers(mods):
    # Large answers (>= 2^18 IDs) copied into the pinned result arena, into
    # pinned caller buffers and into pageable ones all equal the oracle.
    import torch

    Rambo, Oracle = mods
    w = synth.make("document", 0.01, m=1 << 16)
    g, o = build_pair(w, Rambo, Oracle)
    q = w.queries
    rids, roff = o.query_batch("keys", q.data, q.offsets)
    assert int(roff[-1]) >= (1 << 18)
    ids_a, off_a = g.query(q.data, q.offsets, kind="keys")  # pinned result arena
    assert np.array_equal(off_a, roff) and np.array_equal(ids_a, rids)
    for pinned in (True, False):
        ids = torch.zeros(int(roff[-1]) + 7, dtype=torch.int32)
        off = torch.zeros(len(q) + 1, dtype=torch.int64)
        if pinned:
            ids, off = ids.pin_memory(), off.pin_memory()
        n = g.query_into(q.data, q.offsets, ids.numpy().view(np.uint32), off.numpy().view(np.uint64), kind="keys")
        assert n == int(roff[-1])
        assert np.array_equal(off.numpy().view(np.uint64), roff)
        assert np.array_equal(ids.numpy()[:n].view(np.uint32), rids)
    g.close()


def test_id_space_beyond_the_shared_memory_bitmap(mods):
    # K above 4096 * 32 IDs: no per-warp bitmap and no member lists, so the
    # set stage is the staged dense scan (one warp per query even for small
    # batches); results equal the oracle, including queries with more
    # survivors than the staging words hold.
    Rambo, Oracle = mods
    from paper_1910_02611_gb300 import EINVAL, RamboError

    rng = np.random.default_rng(11)
    K, B, R, m, eta = 200_000, 16, 2, 1 << 15, 2
    n_sets = 700  # more than the 256 staging words of a warp
    ids = np.sort(rng.choice(K, n_sets, replace=False)).astype(np.uint64)
    common = rng.integers(0, 1 << 62, 40, dtype=np.uint64)  # keys held by every set
    sets = [np.concatenate([common, rng.integers(0, 1 << 62, int(rng.integers(1, 200)), dtype=np.uint64)])
            for _ in range(n_sets)]
    data = np.concatenate(sets)
    off = np.zeros(n_sets + 1, np.uint64)
    np.cumsum([s.size for s in sets], out=off[1:])
    g = Rambo(K, B, R, m, eta, 3)
    o = Oracle(K, B, R, m, eta, 3)
    g.insert(ids, data, off, kind="keys")
    o.insert_keys_batch(ids, data, off)
    assert_partition_equal(g, o)
    qs = [common[:1], common[:3]]  # every set survives
    for t in range(60):
        s = sets[int(rng.integers(0, n_sets))]
        qs.append(s[rng.choice(s.size, int(rng.integers(1, 4)), replace=False)])
    qs.append(rng.integers(0, 1 << 62, 2, dtype=np.uint64))
    qd = np.concatenate(qs)
    qo = np.zeros(len(qs) + 1, np.uint64)
    np.cumsum([q.size for q in qs], out=qo[1:])
    ids_g, off_g = assert_query_equal(g, o, synth.Collection("keys", qd, qo))
    assert off_g[2] - off_g[1] >= n_sets
    base = g.get_config()
    for stage in (2, 3):
        with pytest.raises(RamboError) as e:
            g.set_config(**{**base, "set_stage": stage})
        assert e.value.code == EINVAL
    g.set_config(**{**base, "warps_per_query": 8})  # no bitmap: stays one warp per query
    assert_query_equal(g, o, synth.Collection("keys", qd, qo))
    g.close()


def test_dense_answers_staged_as_bitmaps(mods):
    # A query whose answer holds more IDs than its K-bit set bitmap has words
    # is staged as the bitmap and expanded by the gather; sparser answers are
    # staged as ID lists.  A batch mixing both (K = 2000: 63 bitmap words, the
    # last one partial) must equal the oracle through the direct call (one
    # warp per query, and a whole block per query for a small batch), the
    # host-output pipeline, device inputs and a captured plan, in every set
    # stage.
    import torch

    Rambo, Oracle = mods
    from paper_1910_02611_gb300 import Plan

    rng = np.random.default_rng(2000)
    K, B, R, m, eta = 2000, 32, 4, 1 << 14, 2
    vocab = rng.integers(0, 1 << 62, 400, dtype=np.uint64)
    pop = 1.0 / np.arange(1, vocab.size + 1) ** 1.1
    pop /= pop.sum()
    ids = np.sort(rng.choice(K, 1900, replace=False)).astype(np.uint64)  # 100 IDs never inserted
    sets = [np.unique(vocab[rng.choice(vocab.size, int(rng.integers(5, 60)), p=pop)]) for _ in ids]
    data = np.concatenate(sets)
    off = np.zeros(ids.size + 1, np.uint64)
    np.cumsum([s.size for s in sets], out=off[1:])
    g = Rambo(K, B, R, m, eta, 5)
    o = Oracle(K, B, R, m, eta, 5)
    g.insert(ids, data, off, kind="keys")
    o.insert_keys_batch(ids, data, off)
    n = 70_000  # above the host pipeline's threshold
    nt = rng.integers(1, 3, n)
    qo = np.zeros(n + 1, np.uint64)
    np.cumsum(nt, out=qo[1:])
    qd = vocab[rng.integers(0, vocab.size, int(qo[-1]))]
    rids, roff = o.query_batch("keys", qd, qo)
    cnt = np.diff(roff.astype(np.int64))
    bw = (K + 31) // 32
    assert (cnt > bw).sum() > 1000 and ((cnt > 0) & (cnt <= bw)).sum() > 1000  # both staging forms occur
    base = g.get_config()
    try:
        # staging 0: bitmaps above 63 IDs; 1: ID lists only; 3: bitmaps above 189 IDs
        for stage, staging in ((0, 0), (1, 0), (2, 0), (3, 0), (0, 1), (2, 3)):
            g.set_config(**{**base, "set_stage": stage, "answer_staging": staging})
            ids_h, off_h = g.query(qd, qo, kind="keys")  # host output: chunked pipeline
            assert np.array_equal(off_h, roff) and np.array_equal(ids_h, rids)
            ids_d, off_d = g.query(torch.from_numpy(qd.view(np.int64)).cuda(),
                                   torch.from_numpy(qo.view(np.int64)).cuda(), kind="keys")
            assert np.array_equal(off_d.cpu().numpy().view(np.uint64), roff)
            assert np.array_equal(ids_d.cpu().numpy().view(np.uint32), rids)
            sub = synth.Collection("keys", qd[: int(qo[6])], qo[:7])  # a block of warps per query
            assert_query_equal(g, o, sub)
    finally:
        g.set_config(**base)
    nq = 5000
    for staging in (0, 1, 3):
        g.set_config(**{**base, "answer_staging": staging})
        plan = Plan(g, "keys", nq, int(qo[nq]), int(roff[nq]) + 1024)
        plan.launch_host(qd[: int(qo[nq])], qo[: nq + 1])
        ids_p, off_p = plan.wait()
        assert np.array_equal(off_p, roff[: nq + 1]) and np.array_equal(ids_p, rids[: int(roff[nq])])
        plan.close()
    g.set_config(**base)
    from paper_1910_02611_gb300 import EINVAL, RamboError

    with pytest.raises(RamboError) as e:
        g.set_config(**{**base, "answer_staging": 65})
    assert e.value.code == EINVAL
    g.close()
