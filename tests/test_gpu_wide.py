"""GPU parity on the paper's own wide layouts, which the register-tiled
query kernel cannot hold and the block-per-query kernel serves: the stacked
whole-genome index of Sec. 5.2 (B = 50000, R = 5) folded over 1, 2 and 3
times (appendix; B = 25000, 12500, 6250), the ClueWeb09 shape of Sec. 5.3
(B = 2e4, R = 4), the largest B (65535) with an ID space beyond the tiled
kernel's shared-memory bitmap, and
more tables than the tiled kernel's eight (R = 12, 16).  Sizes are scaled
down (small m and K) so the oracle finishes in seconds; index bits, the
partition table and every query's ID list must be identical to the oracle's."""
import numpy as np
import pytest

import synth
from tests.parity import assert_index_equal_by_rows, assert_partition_equal, assert_query_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from oracle.oracle import Oracle
    from paper_1910_02611_gb300 import Rambo

    return Rambo, Oracle


def _key_sets(rng, K, lo, hi, pool=20000, shared=0.3):
    """K sets of random 64-bit keys; a share drawn from a common pool so keys
    sit in several sets (multiplicity V > 1), the rest unique."""
    common = rng.integers(0, 1 << 62, pool, dtype=np.uint64)
    sizes = rng.integers(lo, hi + 1, K)
    data = []
    for n in sizes:
        ns = int(n * shared)
        data.append(np.concatenate([rng.choice(common, ns, replace=False),
                                    rng.integers(0, 1 << 62, int(n) - ns, dtype=np.uint64)]))
    off = np.zeros(K + 1, np.uint64)
    np.cumsum(sizes, out=off[1:])
    return synth.Collection("keys", np.concatenate(data), off, np.arange(K, dtype=np.uint64))


def _key_queries(rng, sets, n, max_terms=4):
    """Conjunctive queries: 1..max_terms keys of one random set (so some
    answer is certain), a few mixed with a fresh key (usually empty)."""
    out, off = [], [0]
    for t in range(n):
        s = sets.item(int(rng.integers(len(sets))))
        q = rng.choice(s, int(rng.integers(1, max_terms + 1)), replace=False)
        if t % 5 == 4:
            q = np.append(q, rng.integers(0, 1 << 62, 1, dtype=np.uint64))
        out.append(q)
        off.append(off[-1] + q.size)
    return synth.Collection("keys", np.concatenate(out), np.array(off, np.uint64))


def _build(mods, K, B, R, m, eta, sets, kind="keys", k=31):
    Rambo, Oracle = mods
    g = Rambo(K, B, R, m, eta, 42)
    g.insert(sets.ids, sets.data, sets.offsets, kind=kind, k=k)
    o = Oracle(K, B, R, m, eta, 42)
    if kind == "keys":
        o.insert_keys_batch(sets.ids, sets.data, sets.offsets, nthreads=8)
    else:
        o.insert_seq_batch(sets.ids, sets.data, sets.offsets, k, nthreads=8)
    return g, o


def test_stacked_wgs_shape_b50000_r5_and_its_folds(mods):
    Rambo, Oracle = mods
    rng = np.random.default_rng(50000)
    K, B, R, m, eta = 3000, 50000, 5, 1 << 11, 2
    sets = _key_sets(rng, K, 50, 300)
    g, o = _build(mods, K, B, R, m, eta, sets)
    assert g.info().row_stride == 1564  # 6.25 KB rows
    assert_index_equal_by_rows(g, o)
    assert_partition_equal(g, o)
    q = _key_queries(rng, sets, 300)
    assert_query_equal(g, o, q)
    for f in range(1, 4):  # folding over: B -> B/2 (appendix), three times
        g.fold()
        B2 = B >> f
        of = Oracle(K, B2, R, m, eta, 42)
        of.insert_keys_batch(sets.ids, sets.data, sets.offsets, nthreads=8)
        assert g.B == B2
        assert_index_equal_by_rows(g, of)
        assert_partition_equal(g, of)
        assert_query_equal(g, of, q)
    g.close()


def test_clueweb_shape_b20000_r4_with_sequences_plans_and_baseline(mods):
    import torch

    from paper_1910_02611_gb300 import Plan

    rng = np.random.default_rng(20000)
    w = synth.make("genome", 0.02, m=1 << 12, B=20000, R=4)
    g, o = _build(mods, w.K, 20000, 4, w.m, w.eta, w.sets, kind="seq")
    assert_index_equal_by_rows(g, o)
    q = w.queries.subset(np.arange(400))
    ids, off = assert_query_equal(g, o, q)
    assert off[-1] > 0
    plan = Plan(g, "seq", max_queries=len(q), max_items=int(q.offsets[-1]), max_ids=1 << 20)
    plan.launch_host(q.data, q.offsets)
    pids, poff = plan.wait()
    assert np.array_equal(poff, off) and np.array_equal(pids, ids)
    plan.close()
    sub = q.subset(np.arange(40))
    bids, boff = g.query_one_per_launch(torch.from_numpy(sub.data).cuda(), sub.offsets, kind="seq")
    rids, roff = o.query_batch("seq", sub.data, sub.offsets, k=31)
    assert np.array_equal(boff, roff) and np.array_equal(bids, rids)
    g.close()


@pytest.mark.parametrize("R,B", [(12, 64), (16, 300), (9, 4096)])
def test_more_tables_than_the_tiled_kernel(mods, R, B):
    rng = np.random.default_rng(R * 1000 + B)
    K, m, eta = 1500, 1 << 12, 3
    sets = _key_sets(rng, K, 20, 200)
    g, o = _build(mods, K, B, R, m, eta, sets)
    assert_index_equal_by_rows(g, o)
    assert_partition_equal(g, o)
    assert_query_equal(g, o, _key_queries(rng, sets, 400))
    g.close()


def test_wide_edge_cases(mods):
    # B = 65535 (the largest), K beyond the 2^17 IDs the tiled kernel's
    # shared-memory bitmap holds, an empty query batch, and an insert after
    # queries (registration changes)
    Rambo, Oracle = mods
    rng = np.random.default_rng(65535)
    K, B, R, m, eta = 140_000, 65535, 2, 1 << 8, 1
    sets = _key_sets(rng, 2000, 5, 40)
    sets = synth.Collection("keys", sets.data, sets.offsets, (np.arange(2000, dtype=np.uint64) * 67) % K)
    g, o = _build(mods, K, B, R, m, eta, sets)
    assert_index_equal_by_rows(g, o)
    q = _key_queries(rng, sets, 200, max_terms=2)
    assert_query_equal(g, o, q)
    ids, off = g.query(q.data[:0], np.zeros(1, np.uint64), kind="keys")
    assert off.tolist() == [0] and ids.size == 0
    extra = _key_sets(rng, 10, 5, 20)
    extra = synth.Collection("keys", extra.data, extra.offsets, np.arange(10, dtype=np.uint64) + K - 10)
    g.insert(extra.ids, extra.data, extra.offsets, kind="keys")
    o.insert_keys_batch(extra.ids, extra.data, extra.offsets)
    assert_query_equal(g, o, _key_queries(rng, extra, 50, max_terms=2))
    g.close()
