"""The sequence query that allocates nothing (rambo_query_seq_batch_noalloc).

It serves callers that cannot allocate device memory while they query, e.g.
a serving thread with a fixed memory budget or code running where cudaMalloc
is not allowed: its working memory is a fixed array the library reserves on
each GPU.  Its answers must equal those of the allocating entry point
(rambo_query_seq_batch_into) exactly -- set IDs are integers -- and must not
depend on what an earlier call left in the shared array, so two calls in a
row on different batches are compared.  This file runs last in the suite
(its name sorts last) and also passes on its own in a fresh process."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_query_equals_allocating_query_on_two_calls_in_a_row():
    import torch

    from paper_1910_02611_gb300 import Rambo

    dev = torch.device("cuda")
    w = synth.make("genome", 0.02, m=1 << 18)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq", k=w.k)
    # two different batches: the second call finds the first call's data in the array
    batches = [w.queries.subset(np.arange(0, 700)), w.queries.subset(np.arange(700, 1000))]
    for q in batches:
        qd = torch.from_numpy(q.data).to(dev)
        qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
        ref_ids = torch.empty(1 << 21, dtype=torch.int32, device=dev)
        ref_off = torch.empty(len(q) + 1, dtype=torch.int64, device=dev)
        n_ref = g.query_into(qd, qo, ref_ids, ref_off, kind="seq", k=w.k)
        ids = torch.full((1 << 21,), -1, dtype=torch.int32, device=dev)
        off = torch.full((len(q) + 1,), -1, dtype=torch.int64, device=dev)
        n = g.query_seq_noalloc(qd, qo, ids, off, k=w.k)
        assert n == n_ref
        assert torch.equal(off, ref_off)
        assert torch.equal(ids[:n], ref_ids[:n_ref])
        assert n > 0
    g.close()


def test_noalloc_rejects_requests_beyond_its_fixed_scratch():
    import torch

    from paper_1910_02611_gb300 import E2BIG, ENOSPC, Rambo, RamboError

    dev = torch.device("cuda")
    w = synth.make("genome", 0.01, m=1 << 16)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq", k=w.k)
    too_many = (1 << 19) + 1
    qo = torch.zeros(too_many + 1, dtype=torch.int64, device=dev)
    qd = torch.zeros(1, dtype=torch.uint8, device=dev)
    out = torch.empty(16, dtype=torch.int32, device=dev)
    off = torch.empty(too_many + 1, dtype=torch.int64, device=dev)
    with pytest.raises(RamboError) as e:
        g.query_seq_noalloc(qd, qo, out, off)
    assert e.value.code == E2BIG
    # a batch whose answers do not fit the caller's buffer reports the size needed
    q = w.queries.subset(np.arange(200))
    qd = torch.from_numpy(q.data).to(dev)
    qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
    off = torch.empty(len(q) + 1, dtype=torch.int64, device=dev)
    n_ref = g.query_into(qd, qo, torch.empty(1 << 20, dtype=torch.int32, device=dev), off, kind="seq")
    if n_ref:
        with pytest.raises(RamboError) as e:
            g.query_seq_noalloc(qd, qo, torch.empty(n_ref - 1, dtype=torch.int32, device=dev), off)
        assert e.value.code == ENOSPC
    g.close()


def test_noalloc_large_batch_takes_the_multi_pass_scan():
    # more than 32768 queries: the count scan runs as three kernels over the
    # fixed scan region instead of one block
    import torch

    from paper_1910_02611_gb300 import Rambo

    dev = torch.device("cuda")
    w = synth.make("genome", 0.02, m=1 << 18)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq", k=w.k)
    rng = np.random.default_rng(77)
    q = synth.substring_queries(rng, w.sets, np.full(40_000, 31), max_subst=0.0)
    qd = torch.from_numpy(q.data).to(dev)
    qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
    ref_ids = torch.empty(1 << 22, dtype=torch.int32, device=dev)
    ref_off = torch.empty(len(q) + 1, dtype=torch.int64, device=dev)
    n_ref = g.query_into(qd, qo, ref_ids, ref_off, kind="seq", k=w.k)
    for _ in range(2):
        ids = torch.full((1 << 22,), -1, dtype=torch.int32, device=dev)
        off = torch.full((len(q) + 1,), -1, dtype=torch.int64, device=dev)
        n = g.query_seq_noalloc(qd, qo, ids, off, k=w.k)
        assert n == n_ref and n >= len(q)  # every query is an exact substring: at least its own set
        assert torch.equal(off, ref_off)
        assert torch.equal(ids[:n], ref_ids[:n_ref])
    g.close()


def test_noalloc_reports_e2big_when_staged_answers_exceed_its_limit():
    # an index whose filters are all ones answers every query with every set;
    # such dense answers are staged as K-bit bitmaps (4096 sets: 128 words a
    # query), so 40,000 queries stage 5,120,000 words > the 4,194,304-word limit
    import torch

    from paper_1910_02611_gb300 import E2BIG, Rambo, RamboError

    dev = torch.device("cuda")
    K = 4096
    g = Rambo(K, 64, 2, 1 << 6, 1, 42)
    rng = np.random.default_rng(5)
    sets = synth.random_bases(rng, K * 300)
    off = np.arange(K + 1, dtype=np.uint64) * np.uint64(300)
    g.insert(np.arange(K, dtype=np.uint64), sets, off, kind="seq", k=31)
    nq = 40_000
    qb = synth.random_bases(rng, nq * 31)
    qd = torch.from_numpy(qb).to(dev)
    qo = torch.from_numpy((np.arange(nq + 1, dtype=np.int64) * 31)).to(dev)
    ids = torch.empty(nq * K, dtype=torch.int32, device=dev)
    out_off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    n_ref = g.query_into(qd, qo, ids, out_off, kind="seq", k=31)
    assert n_ref == nq * K
    with pytest.raises(RamboError) as e:
        g.query_seq_noalloc(qd, qo, ids, out_off, k=31)
    assert e.value.code == E2BIG
    # a batch within the limit (32,000 x 128 words) still answers, after the failed call
    n_ok = 32_000
    n = g.query_seq_noalloc(qd[: n_ok * 31], qo[: n_ok + 1], ids, out_off[: n_ok + 1], k=31)
    assert n == n_ok * K
    assert torch.equal(out_off[: n_ok + 1].cpu(), torch.arange(n_ok + 1, dtype=torch.int64) * K)
    assert torch.equal(ids[:n].view(n_ok, K).cpu(), torch.arange(K, dtype=torch.int32).expand(n_ok, K))
    g.close()
