"""Parity at the benchmark's full sizes for the uneven-length workload
(K=10^4 genome-like sets of 2*10^5 31-mers, B=128, R=8, m=2^26, eta=2; one
batch of 10^6 sequences of lognormal length) and the document workload
(K=10^5 documents, B=320, R=8, m=2^25, eta=3; one batch of 10^6 conjunctive
queries of 1-5 terms), each answered as one full batch the way bench.py
times it.  The oracle builds its own full index from the same sets; the GPU
index is checked on every Bloom filter's population count and the answers
on a sample of the batch's queries (compared on the device-side results, so
the 72 GB of document answers never leave the GPU)."""
import os

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
NT = os.cpu_count() or 1


def _check(name, n_sample, seed):
    import torch

    from oracle.oracle import Oracle
    from paper_1910_02611_gb300 import Rambo

    w = synth.make(name, 1.0)
    dev = torch.device("cuda")
    sets = w.sets
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(torch.from_numpy(sets.ids.view(np.int64)).to(dev),
             torch.from_numpy(sets.data.view(np.int64) if sets.kind == "keys" else sets.data).to(dev),
             torch.from_numpy(sets.offsets.view(np.int64)).to(dev), kind=sets.kind, k=w.k)
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    if sets.kind == "keys":
        o.insert_keys_batch(sets.ids, sets.data, sets.offsets, nthreads=NT)
    else:
        o.insert_seq_batch(sets.ids, sets.data, sets.offsets, w.k, nthreads=NT)
    assert np.array_equal(g.cell_popcount(), o.cell_popcount())
    q = w.queries
    qd = torch.from_numpy(q.data.view(np.int64) if q.kind == "keys" else q.data).to(dev)
    qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
    ids, off = g.query(qd, qo, kind=q.kind, k=w.k, copy=False)  # the whole batch, views of the device arena
    sample = np.sort(np.random.default_rng(seed).choice(len(q), n_sample, replace=False))
    sub = q.subset(sample)
    rids, roff = o.query_batch(q.kind, sub.data, sub.offsets, k=w.k, nthreads=NT)
    off_s = off[torch.from_numpy(sample).to(dev)].cpu().numpy().view(np.uint64)
    end_s = off[torch.from_numpy(sample + 1).to(dev)].cpu().numpy().view(np.uint64)
    for t, qi in enumerate(sample):
        got = ids[int(off_s[t]): int(end_s[t])].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, rids[roff[t]: roff[t + 1]]), (name, int(qi))
    g.close()


def test_fullsize_uneven():
    _check("uneven", 2000, 81)


def test_fullsize_document():
    _check("document", 2000, 82)
