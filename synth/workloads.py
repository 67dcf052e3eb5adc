"""Seeded synthetic inputs shaped like the RAMBO paper's workloads.

The paper's data (ENA whole-genome sequences, Sec. 5.2; Wiki dump and
ClueWeb09 documents, Sec. 5.3) is not available, so these generators stand in
for it.  This module holds none of the method's arithmetic (no hashing, no
Bloom filters): it only draws random DNA, random 64-bit term keys and query
lists, and both the GPU library's tests and the CPU oracle consume its output.

Workloads (sizes are the full ones; ``scale`` shrinks the counts):

- ``tiny``: K=100 sets of 10^4 distinct uniform random 31-mers (2-bit packed
  into uint64); B=10, R=3, m=2^20, eta=2; 10^4 single-key queries, half a
  random member of a random set, half a fresh random 31-mer.
- ``genome``: K=2000 genomes of 1000 chunks x 1000 bases; half the chunks come
  from a shared pool of 10^4 chunks picked without repeat with Zipf(1.1)
  popularity, half are fresh random; B=64, R=6, m=2^27, eta=2; 10^5 query
  sequences of U[100,1000] bases, each a substring of a random genome with a
  per-query substitution rate drawn from U[0, 2%].
- ``uneven``: K=10^4 genomes of 200 chunks (same pool); B=128, R=8, m=2^26,
  eta=2; 10^6 query sequences with lognormal lengths (median 300, sigma 1,
  clipped to [31, 10^4]), substitutions as above.
- ``document``: K=10^5 documents over a 10^6-term vocabulary whose keys are
  random distinct uint64 values; a document is a set of distinct terms drawn
  with Zipf(1.0) popularity, its size lognormal with mean 500 (sigma 1);
  B=320, R=8, m=2^25, eta=3; 10^6 conjunctive queries of U{1..5} distinct
  terms drawn by corpus term frequency.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
_CODE = np.full(256, 255, np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _CODE[_c] = _i
    _CODE[ord(chr(_c).lower())] = _i

DATA_SEED_BASE = 1000  # data seed = 1000 + config number
INDEX_SEED = 42


@dataclass
class Collection:
    """CSR batch: item t is data[offsets[t]:offsets[t+1]].

    kind 'keys': data is uint64 keys; kind 'seq': data is ASCII bases (uint8)."""

    kind: str
    data: np.ndarray
    offsets: np.ndarray
    ids: np.ndarray | None = None  # set IDs for inserted collections

    def __len__(self) -> int:
        return int(self.offsets.size - 1)

    def item(self, t: int) -> np.ndarray:
        return self.data[int(self.offsets[t]) : int(self.offsets[t + 1])]

    def subset(self, idx) -> "Collection":
        idx = np.asarray(idx, np.int64)
        lens = (self.offsets[idx + 1] - self.offsets[idx]).astype(np.int64)
        off = np.zeros(idx.size + 1, np.uint64)
        np.cumsum(lens, out=off[1:])
        gather = _ragged_gather(self.offsets[idx].astype(np.int64), lens)
        ids = None if self.ids is None else self.ids[idx].copy()
        return Collection(self.kind, self.data[gather], off, ids)


@dataclass
class Workload:
    name: str
    K: int
    B: int
    R: int
    m: int
    eta: int
    k: int
    seed: int
    sets: Collection
    queries: Collection
    meta: dict = field(default_factory=dict)

    @property
    def params(self) -> dict:
        return dict(K=self.K, B=self.B, R=self.R, m=self.m, eta=self.eta, seed=self.seed)


def _ragged_gather(starts: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Flat indices starts[t] + arange(lens[t]) for every t, concatenated."""
    total = int(lens.sum())
    if total == 0:
        return np.zeros(0, np.int64)
    rep_start = np.repeat(starts - np.concatenate(([0], np.cumsum(lens)[:-1])), lens)
    return rep_start + np.arange(total, dtype=np.int64)


def random_bases(rng: np.random.Generator, n: int) -> np.ndarray:
    return ACGT[np.frombuffer(rng.bytes(n), np.uint8) & 3]


def random_kmers(rng: np.random.Generator, n: int, k: int = 31) -> np.ndarray:
    """n uniform random k-mers as 2-bit packed uint64 values."""
    bits = 2 * k
    v = rng.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)
    if bits < 64:
        v &= np.uint64((1 << bits) - 1)
    return v


# ----------------------------------------------------------------------------
# config 1: tiny
# ----------------------------------------------------------------------------

def tiny(scale: float = 1.0, n_sets: int = 100, set_size: int = 10_000, n_queries: int = 10_000,
         B: int = 10, R: int = 3, m: int = 1 << 20, eta: int = 2, data_seed: int = DATA_SEED_BASE + 1) -> Workload:
    rng = np.random.default_rng(data_seed)
    n_sets = max(1, int(round(n_sets * scale))) if scale != 1.0 else n_sets
    set_size = max(1, int(round(set_size * scale))) if scale != 1.0 else set_size
    n_queries = max(1, int(round(n_queries * scale))) if scale != 1.0 else n_queries
    keys = []
    for _ in range(n_sets):
        s = np.unique(random_kmers(rng, set_size))
        while s.size < set_size:
            s = np.unique(np.concatenate([s, random_kmers(rng, set_size - s.size)]))
        keys.append(rng.permutation(s))
    data = np.concatenate(keys)
    off = np.arange(n_sets + 1, dtype=np.uint64) * np.uint64(set_size)
    sets = Collection("keys", data, off, np.arange(n_sets, dtype=np.uint64))
    n_in = n_queries // 2
    qs = rng.integers(0, n_sets, n_in)
    qi = rng.integers(0, set_size, n_in)
    member = data[qs * set_size + qi]
    fresh = random_kmers(rng, n_queries - n_in)
    q = np.concatenate([member, fresh])
    perm = rng.permutation(q.size)
    queries = Collection("keys", q[perm], np.arange(q.size + 1, dtype=np.uint64))
    return Workload("tiny", n_sets, B, R, m, eta, 31, INDEX_SEED, sets, queries,
                    meta=dict(member_query=(perm < n_in)))


# ----------------------------------------------------------------------------
# configs 2, 3: genome-like
# ----------------------------------------------------------------------------

def _zipf_pick_without_repeat(rng, n_pool: int, n_pick: int, n_rows: int, s: float) -> np.ndarray:
    """Rows of n_pick distinct pool indices, drawn by successive sampling with
    weight (rank+1)^-s (Gumbel top-k, which is exactly that distribution)."""
    logw = -s * np.log(np.arange(1, n_pool + 1, dtype=np.float64))
    out = np.empty((n_rows, n_pick), np.int64)
    step = max(1, int(4_000_000 // max(n_pool, 1)))
    for a in range(0, n_rows, step):
        b = min(n_rows, a + step)
        g = logw[None, :] + rng.gumbel(size=(b - a, n_pool))
        out[a:b] = np.argpartition(-g, n_pick - 1, axis=1)[:, :n_pick]
    return out


def genomes(rng, n_sets: int, chunks_per_genome: int, chunk_len: int, pool_chunks: int,
            zipf_s: float = 1.1, shared_frac: float = 0.5) -> Collection:
    """Synthetic genomes: chunks drawn half from a shared Zipf-popular pool
    (without repeat inside a genome) and half fresh random, in random order."""
    pool = random_bases(rng, pool_chunks * chunk_len).reshape(pool_chunks, chunk_len)
    n_shared = int(round(chunks_per_genome * shared_frac))
    n_shared = min(n_shared, pool_chunks)
    n_fresh = chunks_per_genome - n_shared
    glen = chunks_per_genome * chunk_len
    data = np.empty(n_sets * glen, np.uint8)
    block = max(1, (64 << 20) // max(glen, 1))
    for a in range(0, n_sets, block):
        b = min(n_sets, a + block)
        g = b - a
        picks = _zipf_pick_without_repeat(rng, pool_chunks, n_shared, g, zipf_s) if n_shared else np.zeros((g, 0), np.int64)
        chunks = np.empty((g, chunks_per_genome, chunk_len), np.uint8)
        chunks[:, :n_shared] = pool[picks]
        chunks[:, n_shared:] = random_bases(rng, g * n_fresh * chunk_len).reshape(g, n_fresh, chunk_len)
        perm = np.argsort(rng.random((g, chunks_per_genome)), axis=1)
        chunks = np.take_along_axis(chunks, perm[:, :, None], axis=1)
        data[a * glen : b * glen] = chunks.reshape(-1)
    off = np.arange(n_sets + 1, dtype=np.uint64) * np.uint64(glen)
    return Collection("seq", data, off, np.arange(n_sets, dtype=np.uint64))


def substring_queries(rng, sets: Collection, lengths: np.ndarray, max_subst: float = 0.02) -> Collection:
    """Each query: a substring of a uniform random set's sequence, with every
    base substituted (to a uniform other base) with a per-query probability
    drawn from U[0, max_subst]."""
    n = lengths.size
    set_len = (sets.offsets[1:] - sets.offsets[:-1]).astype(np.int64)
    g = rng.integers(0, len(sets), n)
    lengths = np.minimum(lengths.astype(np.int64), set_len[g])
    starts = (rng.random(n) * (set_len[g] - lengths + 1)).astype(np.int64) + sets.offsets[g].astype(np.int64)
    idx = _ragged_gather(starts, lengths)
    q = sets.data[idx].copy()
    rate = rng.random(n) * max_subst
    per_base_rate = np.repeat(rate, lengths)
    hit = rng.random(q.size) < per_base_rate
    codes = _CODE[q[hit]].astype(np.int64)
    q[hit] = ACGT[(codes + rng.integers(1, 4, codes.size)) & 3]
    off = np.zeros(n + 1, np.uint64)
    np.cumsum(lengths, out=off[1:])
    return Collection("seq", q, off)


def genome(scale: float = 1.0, data_seed: int = DATA_SEED_BASE + 2, *, n_sets=2000, chunks_per_genome=1000,
           chunk_len=1000, pool_chunks=10_000, n_queries=100_000, qlen=(100, 1000),
           B=64, R=6, m=1 << 27, eta=2) -> Workload:
    rng = np.random.default_rng(data_seed)
    if scale != 1.0:
        n_sets = max(2, int(round(n_sets * scale)))
        chunks_per_genome = max(2, int(round(chunks_per_genome * scale)))
        pool_chunks = max(chunks_per_genome, int(round(pool_chunks * scale)))
        n_queries = max(1, int(round(n_queries * scale)))
    sets = genomes(rng, n_sets, chunks_per_genome, chunk_len, pool_chunks)
    lengths = rng.integers(qlen[0], qlen[1] + 1, n_queries)
    queries = substring_queries(rng, sets, lengths)
    return Workload("genome", n_sets, B, R, m, eta, 31, INDEX_SEED, sets, queries)


def uneven(scale: float = 1.0, data_seed: int = DATA_SEED_BASE + 3, *, n_sets=10_000, chunks_per_genome=200,
           chunk_len=1000, pool_chunks=10_000, n_queries=1_000_000, median=300.0, sigma=1.0,
           qlen_clip=(31, 10_000), B=128, R=8, m=1 << 26, eta=2) -> Workload:
    rng = np.random.default_rng(data_seed)
    if scale != 1.0:
        n_sets = max(2, int(round(n_sets * scale)))
        chunks_per_genome = max(2, int(round(chunks_per_genome * scale)))
        pool_chunks = max(chunks_per_genome, int(round(pool_chunks * scale)))
        n_queries = max(1, int(round(n_queries * scale)))
    sets = genomes(rng, n_sets, chunks_per_genome, chunk_len, pool_chunks)
    lengths = np.clip(np.round(rng.lognormal(np.log(median), sigma, n_queries)), qlen_clip[0], qlen_clip[1]).astype(np.int64)
    queries = substring_queries(rng, sets, lengths)
    return Workload("uneven", n_sets, B, R, m, eta, 31, INDEX_SEED, sets, queries)


# ----------------------------------------------------------------------------
# config 4: documents
# ----------------------------------------------------------------------------

def _distinct_by_weight(rng, cdf: np.ndarray, n: int) -> np.ndarray:
    """n distinct indices by successive sampling with the given weights."""
    n = min(n, cdf.size)
    got = np.zeros(0, np.int64)
    order = np.zeros(0, np.int64)
    draw = max(8, int(n * 1.6))
    while got.size < n:
        x = np.searchsorted(cdf, rng.random(draw) * cdf[-1], side="right")
        allx = np.concatenate([order, x])
        u, first = np.unique(allx, return_index=True)
        order = allx[np.sort(first)]
        got = order
        draw = max(8, 2 * (n - got.size) + 16)
    return got[:n]


def documents(scale: float = 1.0, data_seed: int = DATA_SEED_BASE + 4, *, n_docs=100_000, vocab=1_000_000,
              mean_len=500.0, sigma=1.0, zipf_s=1.0, n_queries=1_000_000, qterms=(1, 5),
              B=320, R=8, m=1 << 25, eta=3) -> Workload:
    rng = np.random.default_rng(data_seed)
    if scale != 1.0:
        n_docs = max(2, int(round(n_docs * scale)))
        vocab = max(1000, int(round(vocab * scale)))
        n_queries = max(1, int(round(n_queries * scale)))
    keys = np.unique(rng.integers(0, np.iinfo(np.uint64).max, size=int(vocab * 1.01) + 16, dtype=np.uint64, endpoint=True))
    keys = rng.permutation(keys)[:vocab]
    w = np.arange(1, vocab + 1, dtype=np.float64) ** (-zipf_s)
    cdf = np.cumsum(w)
    mu = np.log(mean_len) - sigma * sigma / 2
    lens = np.clip(np.round(rng.lognormal(mu, sigma, n_docs)), 1, vocab).astype(np.int64)
    terms = [_distinct_by_weight(rng, cdf, int(L)) for L in lens]
    tid = np.concatenate(terms)
    off = np.zeros(n_docs + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    sets = Collection("keys", keys[tid], off, np.arange(n_docs, dtype=np.uint64))
    df = np.bincount(tid, minlength=vocab).astype(np.float64)
    dcdf = np.cumsum(df)
    nt = rng.integers(qterms[0], qterms[1] + 1, n_queries)
    q = np.searchsorted(dcdf, rng.random((n_queries, qterms[1])) * dcdf[-1], side="right")
    # redraw repeated terms inside a query until its first nt terms are distinct
    for _ in range(100):
        srt = np.sort(q, axis=1)
        dup_any = np.zeros(n_queries, bool)
        for a in range(qterms[1]):
            for b in range(a + 1, qterms[1]):
                dup_any |= (q[:, a] == q[:, b]) & (b < nt)
        if not dup_any.any():
            break
        rows = np.nonzero(dup_any)[0]
        q[rows] = np.searchsorted(dcdf, rng.random((rows.size, qterms[1])) * dcdf[-1], side="right")
        del srt
    mask = np.arange(qterms[1])[None, :] < nt[:, None]
    qoff = np.zeros(n_queries + 1, np.uint64)
    np.cumsum(nt, out=qoff[1:])
    queries = Collection("keys", keys[q[mask]], qoff)
    return Workload("document", n_docs, B, R, m, eta, 31, INDEX_SEED, sets, queries,
                    meta=dict(vocab_keys=keys, df=df))


GENERATORS = {"tiny": tiny, "genome": genome, "uneven": uneven, "document": documents}


def make(name: str, scale: float = 1.0, **kw) -> Workload:
    return GENERATORS[name](scale=scale, **kw)
