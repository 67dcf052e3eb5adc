"""The seeded synthetic workloads have the shapes the measurements are quoted
on: k-mer sets and query mixes (tiny), genomes of shared Zipf-popular and
fresh chunks with substring queries (genome, uneven), lognormal documents of
distinct Zipf terms with 1-5-term queries drawn by document frequency
(document).  CPU only, on scaled-down instances."""
import numpy as np

import synth


def test_tiny_sets_and_query_mix():
    w = synth.make("tiny", 1.0)
    assert (w.K, w.B, w.R, w.m, w.eta) == (100, 10, 3, 1 << 20, 2)
    sizes = np.diff(w.sets.offsets.astype(np.int64))
    assert np.all(sizes == 10_000)
    for t in range(0, 100, 17):
        s = w.sets.item(t)
        assert np.unique(s).size == s.size  # distinct k-mers
        assert int(s.max()) < 4 ** 31       # 31-mers, 2 bits a base
    q = w.queries.data
    member = w.meta["member_query"]
    assert len(w.queries) == 10_000 and member.sum() == 5_000
    allk = np.unique(w.sets.data)
    assert np.isin(q[member], allk).all()
    assert np.isin(q[~member], allk).mean() < 0.01  # fresh random k-mers


def test_genome_chunks_shared_and_fresh():
    w = synth.make("genome", 0.02)
    assert (w.B, w.R, w.m, w.eta, w.k) == (64, 6, 1 << 27, 2, 31)
    n, glen = len(w.sets), int(w.sets.offsets[1])
    chunks = w.sets.data.reshape(n, glen // 1000, 1000)
    assert set(np.unique(w.sets.data)) <= set(b"ACGT")
    # a chunk occurs in several genomes iff it came from the shared pool
    view = np.ascontiguousarray(chunks).view(np.dtype((np.void, 1000))).reshape(n, -1)
    uniq, counts = np.unique(view.ravel(), return_counts=True)
    in_many = counts > 1
    per_genome_shared = np.array([np.isin(view[g], uniq[in_many]).sum() for g in range(n)])
    half = chunks.shape[1] // 2
    assert np.all(per_genome_shared <= half)
    assert per_genome_shared.mean() > 0.5 * half  # most pool chunks recur
    assert counts.max() >= n // 2                 # Zipf head: a chunk shared by many genomes
    lens = np.diff(w.queries.offsets.astype(np.int64))
    assert lens.min() >= 100 and lens.max() <= 1000


def test_substring_queries_with_bounded_substitutions():
    rng = np.random.default_rng(5)
    sets = synth.genomes(rng, 4, 20, 1000, 30)
    lengths = rng.integers(100, 1001, 200)
    # recover each query's source by brute force on this small collection
    q = synth.substring_queries(np.random.default_rng(6), sets, lengths)
    seqs = [sets.item(t) for t in range(len(sets))]
    for i in range(0, 200, 20):
        x = q.item(i)
        best = min(int(np.count_nonzero(np.lib.stride_tricks.sliding_window_view(s, x.size) != x, axis=1).min())
                   for s in seqs)
        assert best <= 0.02 * x.size + 4 * np.sqrt(0.02 * x.size) + 1


def test_uneven_lengths_lognormal_and_clipped():
    w = synth.make("uneven", 0.002, n_queries=2_500_000)  # 5000 queries at this scale
    assert (w.B, w.R, w.m, w.eta) == (128, 8, 1 << 26, 2)
    lens = np.diff(w.queries.offsets.astype(np.int64))
    assert lens.size == 5000
    assert lens.min() >= 31 and lens.max() <= 10_000
    assert 250 <= np.median(lens) <= 350
    assert np.std(np.log(lens)) > 0.8  # lognormal spread (sigma 1, clipped at the ends)


def test_documents_lengths_terms_and_queries():
    w = synth.make("document", 0.01)
    assert (w.B, w.R, w.m, w.eta) == (320, 8, 1 << 25, 3)
    lens = np.diff(w.sets.offsets.astype(np.int64))
    assert 400 <= lens.mean() <= 600  # lognormal with mean 500
    for t in range(0, len(w.sets), 97):
        d = w.sets.item(t)
        assert np.unique(d).size == d.size  # distinct terms
    nt = np.diff(w.queries.offsets.astype(np.int64))
    assert nt.min() == 1 and nt.max() == 5
    assert np.all(np.bincount(nt)[1:] > 0.15 * nt.size)  # U{1..5}
    for i in range(0, len(w.queries), 211):
        x = w.queries.item(i)
        assert np.unique(x).size == x.size
    # terms drawn by document frequency: each frequent term's share of the query
    # terms is its share of all (document, term) pairs, within sampling error
    df = w.meta["df"]
    keys = w.meta["vocab_keys"]
    n_terms = w.queries.data.size
    for rank in range(5):
        t = np.argsort(-df)[rank]
        want = n_terms * df[t] / df.sum()
        got = np.count_nonzero(w.queries.data == keys[t])
        assert abs(got - want) <= 5 * np.sqrt(want) + 2, (rank, got, want)
