"""Graph-captured plans and the continuous-batching server, against the CPU
oracle.

- A plan replays one captured CUDA graph for batches of any size up to its
  capacity; every batch must equal the plain query call and the oracle.
- The server batches requests as they arrive over several in-flight slots and
  applies streaming inserts (Sec. 3.1) as ordering barriers.  Every answer must
  equal the oracle's at that point of the request stream, and be the same
  whether the request rode in a mixed batch or was submitted alone."""
import numpy as np
import pytest

import synth
from tests.parity import assert_query_equal

pytestmark = pytest.mark.gpu


def _mods():
    from oracle.oracle import Oracle
    from paper_1910_02611_gb300 import Plan, Rambo, Server

    return Rambo, Oracle, Plan, Server


def test_plan_replays_match_query_calls():
    import torch

    from paper_1910_02611_gb300 import E2BIG, EINVAL, RamboError

    Rambo, Oracle, Plan, _ = _mods()
    w = synth.make("genome", 0.02, m=1 << 18)
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(w.sets.ids, w.sets.data, w.sets.offsets, kind="seq")
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31)
    plan = Plan(g, "seq", max_queries=600, max_items=600 * 1000, max_ids=1 << 20)
    # intake (validation + packing), the two query-kernel instances, one-block
    # scan, gather: five kernels per replay (the status reset rides on the
    # descriptor copy)
    assert plan.launches_per_replay == 5
    rng = np.random.default_rng(3)
    for n, timed in ((1, True), (37, False), (600, True), (250, False), (250, True)):
        # the graph with timing nodes reports the query kernel's time; the
        # one without them reports none; both answer the same
        plan.set_timing(timed)
        idx = rng.choice(len(w.queries), n, replace=False)
        q = w.queries.subset(idx)
        plan.launch_host(q.data, q.offsets)
        ids, off = plan.wait(to_host=True)
        rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)
        st = plan.last_stats()
        assert (st["query_kernel_ms"] > 0) == timed and (st["device_ms"] > 0) == timed
        assert st["n_results"] == int(roff[-1]) and st["n_queries"] == n
    with pytest.raises(RamboError) as e:
        plan.set_timing(2)
    assert e.value.code == EINVAL
    # device-side inputs written straight into the plan's buffers
    q = w.queries.subset(np.arange(100))
    dd = torch.from_numpy(q.data).cuda()
    do = torch.from_numpy(q.offsets.view(np.int64)).cuda()
    nbytes = q.data.size
    from paper_1910_02611_gb300.rambo import _CudaArray

    dst = torch.as_tensor(_CudaArray(plan.dev_data_ptr, nbytes, "|u1"), device="cuda")
    dst.copy_(dd)
    dst_off = torch.as_tensor(_CudaArray(plan.dev_offsets_ptr, 101, "<i8"), device="cuda")
    dst_off.copy_(do)
    plan.launch_device(100, nbytes)
    ids, off = plan.wait(to_host=False)
    rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), roff)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), rids)
    # beyond capacity, and offsets not starting at zero
    big = w.queries.subset(np.arange(601))
    with pytest.raises(RamboError) as e:
        plan.launch_host(big.data, big.offsets)
    assert e.value.code == E2BIG
    plan.host_offsets[:3] = [5, 50, 120]
    from paper_1910_02611_gb300.rambo import load_library

    assert load_library().rambo_plan_launch(plan._p, 2, 120, 1, None) == 0
    with pytest.raises(RamboError) as e:
        plan.wait()
    assert e.value.code == EINVAL
    # an unresolved base: EBADSEQ (found by the query kernel from the packing
    # kernel's lowest bad position); the next batch starts from a clean status
    from paper_1910_02611_gb300 import EBADSEQ

    q = w.queries.subset(np.arange(20))
    bad = q.data.copy()
    bad[int(q.offsets[13]) + 5] = ord("N")
    plan.launch_host(bad, q.offsets)
    with pytest.raises(RamboError) as e:
        plan.wait()
    assert e.value.code == EBADSEQ
    plan.launch_host(q.data, q.offsets)
    ids, off = plan.wait()
    rids, roff = o.query_batch("seq", q.data, q.offsets, k=31)
    assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    plan.close()
    # the plain call still agrees afterwards
    assert_query_equal(g, o, w.queries.subset(np.arange(200)))


def _serving_setup(seed=5):
    """Documents (keys) and genomes (DNA) in one index, with spare capacity for
    streamed documents."""
    rng = np.random.default_rng(seed)
    docs = synth.make("document", 0.004, m=1 << 16)
    gen = synth.make("genome", 0.01, m=1 << 16)
    n_docs, n_gen, n_new = len(docs.sets), len(gen.sets), 60
    K = n_docs + n_gen + n_new
    params = dict(K=K, B=docs.B, R=docs.R, m=docs.m, eta=docs.eta, seed=42)
    vocab = docs.meta["vocab_keys"]
    new_docs = []
    for t in range(n_new):
        L = int(rng.integers(20, 200))
        new_docs.append(rng.choice(vocab, L, replace=False))
    return rng, docs, gen, params, n_docs, n_gen, new_docs


def _request_stream(rng, docs, gen, n_docs, n_gen, new_docs, n_req=900):
    """A mixed stream: 1-term and 5-term key queries, DNA sequences of 31..600
    bases, and insert batches of new documents every ~150 requests."""
    ops = []
    vocab = docs.meta["vocab_keys"]
    df = docs.meta["df"]
    p = df / df.sum()
    ins_at = set(range(150, n_req, 150))
    nxt = 0
    for i in range(n_req):
        if i in ins_at and nxt < len(new_docs):
            batch = new_docs[nxt: nxt + 20]
            ids = np.arange(n_docs + n_gen + nxt, n_docs + n_gen + nxt + len(batch), dtype=np.uint64)
            off = np.zeros(len(batch) + 1, np.uint64)
            np.cumsum([b.size for b in batch], out=off[1:])
            ops.append(("insert", ids, np.concatenate(batch).astype(np.uint64), off))
            nxt += len(batch)
        r = rng.random()
        if r < 0.33:
            ops.append(("keys", vocab[rng.choice(vocab.size, 1, p=p)].astype(np.uint64)))
        elif r < 0.66:
            ops.append(("keys", vocab[rng.choice(vocab.size, 5, replace=False, p=p)].astype(np.uint64)))
        else:
            gi = int(rng.integers(0, n_gen))
            s = gen.sets.item(gi)
            L = int(rng.integers(31, 601))
            a = int(rng.integers(0, s.size - L + 1))
            ops.append(("seq", s[a: a + L].copy()))
    return ops


def _oracle_answers(Oracle, params, docs, gen, n_docs, ops):
    o = Oracle(params["K"], params["B"], params["R"], params["m"], params["eta"], params["seed"])
    o.insert_keys_batch(docs.sets.ids, docs.sets.data, docs.sets.offsets)
    o.insert_seq_batch(gen.sets.ids + np.uint64(n_docs), gen.sets.data, gen.sets.offsets, 31)
    want = []
    for op in ops:
        if op[0] == "insert":
            o.insert_keys_batch(op[1], op[2], op[3])
            want.append(None)
        elif op[0] == "keys":
            want.append(o.query_keys(op[1]))
        else:
            want.append(o.query_seq(op[1], 31))
    return want


def _gpu_index(Rambo, params, docs, gen, n_docs):
    g = Rambo(params["K"], params["B"], params["R"], params["m"], params["eta"], params["seed"])
    g.insert(docs.sets.ids, docs.sets.data, docs.sets.offsets, kind="keys")
    g.insert(gen.sets.ids + np.uint64(n_docs), gen.sets.data, gen.sets.offsets, kind="seq")
    return g


def _serve(Server, g, ops, alone: bool, slots=3, max_batch_queries=64):
    srv = Server(g, slots=slots, max_batch_queries=max_batch_queries, max_batch_bases=64 * 700,
                 max_batch_keys=64 * 5, max_batch_ids=1 << 20)
    got = [None] * len(ops)
    tickets = []
    for i, op in enumerate(ops):
        if op[0] == "insert":
            t = srv.submit_insert(op[1], op[2], op[3], kind="keys")
        else:
            t = srv.submit(op[1], kind=op[0])
        tickets.append(t)
        if alone:
            r = srv.result(t)
            got[i] = None if op[0] == "insert" else r[0]
    if not alone:
        srv.drain()
        for i, (op, t) in enumerate(zip(ops, tickets)):
            r = srv.result(t)
            got[i] = None if op[0] == "insert" else r[0]
    st = srv.stats()
    srv.close()
    return got, st


def test_server_answers_equal_oracle_and_are_the_same_alone_and_in_the_mix():
    Rambo, Oracle, _, Server = _mods()
    rng, docs, gen, params, n_docs, n_gen, new_docs = _serving_setup()
    ops = _request_stream(rng, docs, gen, n_docs, n_gen, new_docs)
    want = _oracle_answers(Oracle, params, docs, gen, n_docs, ops)
    g1 = _gpu_index(Rambo, params, docs, gen, n_docs)
    mixed, st_mixed = _serve(Server, g1, ops, alone=False)
    g2 = _gpu_index(Rambo, params, docs, gen, n_docs)
    alone, st_alone = _serve(Server, g2, ops, alone=True)
    n_q = sum(op[0] != "insert" for op in ops)
    for i, op in enumerate(ops):
        if op[0] == "insert":
            continue
        assert np.array_equal(mixed[i], want[i]), (i, op[0])
        assert np.array_equal(alone[i], want[i]), (i, op[0])
    assert st_mixed["queries"] == n_q and st_alone["queries"] == n_q
    assert st_mixed["inserts"] == st_alone["inserts"] == sum(op[0] == "insert" for op in ops)
    # mixed submission really batches; alone submission does not
    assert st_mixed["batches"] < n_q
    assert st_alone["batches"] == n_q
    assert st_mixed["p99_ns"] >= st_mixed["p50_ns"] > 0


def test_server_replay_load_generator():
    Rambo, Oracle, _, Server = _mods()
    rng, docs, gen, params, n_docs, n_gen, new_docs = _serving_setup(seed=9)
    ops = [op for op in _request_stream(rng, docs, gen, n_docs, n_gen, new_docs, n_req=400) if op[0] != "insert"]
    want = _oracle_answers(Oracle, params, docs, gen, n_docs, ops)
    g = _gpu_index(Rambo, params, docs, gen, n_docs)
    srv = Server(g, slots=2, max_batch_queries=32, max_batch_bases=32 * 700, max_batch_keys=32 * 5,
                 max_batch_ids=1 << 20)
    kinds = np.array([0 if op[0] == "keys" else 1 for op in ops], np.uint8)
    payload = [op[1].view(np.uint8) for op in ops]
    boff = np.zeros(len(ops) + 1, np.uint64)
    np.cumsum([p.size for p in payload], out=boff[1:])
    arrivals = np.cumsum(rng.exponential(1e9 / 20000, len(ops))).astype(np.uint64)  # Poisson, 20k/s
    tickets = srv.replay(kinds, np.concatenate(payload), boff, arrivals)
    srv.drain()
    for i, t in enumerate(tickets):
        ids, lat = srv.result(int(t))
        assert np.array_equal(ids, want[i])
    assert srv.stats()["queries"] == len(ops)
    srv.close()


def test_server_requeues_batches_whose_answers_overflow_the_slot():
    # A batch whose answers exceed max_batch_ids is re-run query by query;
    # a query whose own answer exceeds it gets RAMBO_E2BIG.  Every other
    # answer still equals the oracle's.
    from paper_1910_02611_gb300 import E2BIG, RamboError

    Rambo, Oracle, _, Server = _mods()
    rng, docs, gen, params, n_docs, n_gen, new_docs = _serving_setup(seed=13)
    ops = [op for op in _request_stream(rng, docs, gen, n_docs, n_gen, new_docs, n_req=200) if op[0] != "insert"]
    want = _oracle_answers(Oracle, params, docs, gen, n_docs, ops)
    sizes = np.array([w.size for w in want])
    cap = int(max(64, np.percentile(sizes, 80)))  # most single answers fit, most batches do not
    g = _gpu_index(Rambo, params, docs, gen, n_docs)
    srv = Server(g, slots=2, max_batch_queries=64, max_batch_bases=64 * 700, max_batch_keys=64 * 5,
                 max_batch_ids=cap)
    tickets = [srv.submit(op[1], kind=op[0]) for op in ops]
    srv.drain()
    n_big = 0
    for i, t in enumerate(tickets):
        if sizes[i] > cap:
            n_big += 1
            with pytest.raises(RamboError) as e:
                srv.result(int(t))
            assert e.value.code == E2BIG
        else:
            ids, _ = srv.result(int(t))
            assert np.array_equal(ids, want[i]), i
    assert 0 < n_big < len(ops)
    srv.close()


def test_server_defers_batches_when_pinned_memory_is_refused():
    # Pinned host memory for a batch's answers refused (injected on the host:
    # the next n allocations fail as if cudaMallocHost had): the batch's
    # queries are requeued and answered later, identically; a query refused
    # 64 times fails with RAMBO_ENOMEM; the server keeps serving afterwards.
    from paper_1910_02611_gb300 import ENOMEM, RamboError

    Rambo, _, _, Server = _mods()
    rng = np.random.default_rng(9)
    K = 70_000  # every answer alone (70000 IDs, 280 KB) goes to the pinned pool
    g = Rambo(K, 64, 2, 1 << 6, 1, 42)  # tiny filters: every key hits every set
    keys = rng.integers(0, 1 << 62, K * 40, dtype=np.uint64)
    g.insert(np.arange(K, dtype=np.uint64), keys, np.arange(K + 1, dtype=np.uint64) * np.uint64(40), kind="keys")
    want, _ = g.query(keys[:1], np.array([0, 1], np.uint64), kind="keys")
    assert want.size == K
    srv = Server(g, slots=1, max_batch_queries=64, max_batch_bases=0, max_batch_keys=64, max_batch_ids=1 << 23)
    try:
        srv.inject_alloc_failures(3)
        tickets = [srv.submit(keys[i: i + 1], kind="keys") for i in range(200)]
        for t in tickets:
            ids, _ = srv.result(t)
            assert np.array_equal(ids, want)
        assert srv.stats()["deferred"] >= 1
        srv.inject_alloc_failures(1_000_000)
        tickets = [srv.submit(keys[i: i + 1], kind="keys") for i in range(40)]
        for t in tickets:
            with pytest.raises(RamboError) as e:
                srv.result(t)
            assert e.value.code == ENOMEM
        srv.inject_alloc_failures(0)
        tickets = [srv.submit(keys[i: i + 1], kind="keys") for i in range(40)]
        for t in tickets:
            ids, _ = srv.result(t)
            assert np.array_equal(ids, want)
    finally:
        srv.close()
        g.close()
