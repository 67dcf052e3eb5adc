"""Parity at the benchmark's full size, in the launch configuration bench.py
times (genome-like workload: K=2000 genomes of ~10^6 31-mers, B=64, R=6,
m=2^27, eta=2; one batch of 10^5 query sequences).

The oracle builds its own full index from the same synthetic genomes (B*R
separate Bloom filters, Algorithm 1), then the GPU index is checked on every
Bloom filter's population count, on rows sampled from every table (all B cell
bits of each sampled position), and on the ID lists of a sample of the timed
batch's queries answered inside the full batch."""
import os

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full_genome():
    import torch

    from oracle.oracle import Oracle
    from paper_1910_02611_gb300 import Rambo

    w = synth.make("genome", 1.0)
    dev = torch.device("cuda")
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    g.insert(torch.from_numpy(w.sets.ids.view(np.int64)).to(dev), torch.from_numpy(w.sets.data).to(dev),
             torch.from_numpy(w.sets.offsets.view(np.int64)).to(dev), kind="seq")
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31, nthreads=os.cpu_count() or 1)
    yield w, g, o
    g.close()


def test_fullsize_cell_popcounts(full_genome):
    w, g, o = full_genome
    assert np.array_equal(g.cell_popcount(), o.cell_popcount())


def test_fullsize_sampled_rows(full_genome):
    w, g, o = full_genome
    rows = g.export_index()  # [R, m, S]
    rng = np.random.default_rng(77)
    for r in range(w.R):
        for p in rng.integers(0, w.m, 4000):
            want = o.get_row(r, int(p))  # cells as bits of uint64 words
            got = rows[r, p, : (w.B + 31) // 32].astype(np.uint64)
            got64 = np.zeros(want.size, np.uint64)
            for wi in range(got.size):
                got64[wi // 2] |= got[wi] << np.uint64(32 * (wi % 2))
            assert np.array_equal(got64, want), (r, int(p))


def test_fullsize_sampled_queries_in_the_full_batch(full_genome):
    import torch

    w, g, o = full_genome
    q = w.queries
    dev = torch.device("cuda")
    qd = torch.from_numpy(q.data).to(dev)
    qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
    ids, off = g.query(qd, qo, kind="seq")  # the whole batch, as timed
    ids = ids.cpu().numpy().view(np.uint32)
    off = off.cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(78)
    sample = np.sort(rng.choice(len(q), 3000, replace=False))
    sub = q.subset(sample)
    rids, roff = o.query_batch("seq", sub.data, sub.offsets, k=31, nthreads=os.cpu_count() or 1)
    for t, qi in enumerate(sample):
        assert np.array_equal(ids[off[qi]: off[qi + 1]], rids[roff[t]: roff[t + 1]]), int(qi)
