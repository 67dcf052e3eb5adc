"""Pins for the oracle's Algorithm 1 / Algorithm 2 (Secs. 2-4).

Nothing here compares the oracle with itself: it is checked against brute
force over Python sets, special cases that reduce to a single textbook Bloom
filter, exact set identities the algorithm must satisfy, and the paper's
false-positive analysis (Sec. 2 formula, Lemma 4.1, Lemma 4.2).
"""
import numpy as np
import pytest

from oracle.brute import exact_cell_rambo, exact_msmt

M64 = (1 << 64) - 1


def _random_sets(rng, K, lo, hi, shared_pool=0, shared_per_set=0):
    pool = [int(v) for v in rng.integers(0, 1 << 62, shared_pool, dtype=np.uint64)]
    sets = {}
    for i in range(K):
        n = int(rng.integers(lo, hi + 1))
        own = {int(v) for v in rng.integers(0, 1 << 62, n, dtype=np.uint64)}
        if shared_pool:
            own |= {pool[t] for t in rng.choice(shared_pool, shared_per_set, replace=False)}
        sets[i] = own
    return sets, pool


def _build(oracle_mod, sets, K, B, R, m, eta, seed, order=None):
    o = oracle_mod.Oracle(K, B, R, m, eta, seed)
    for i in (order if order is not None else sorted(sets)):
        o.insert_keys(i, np.array(sorted(sets[i]), np.uint64))
    return o


# --------------------------------------------------------------------------
# brute force on tiny inputs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("B,R", [(4, 3), (5, 2), (3, 5)])
def test_equals_exact_cell_rambo_when_filters_are_exact(oracle_mod, B, R):
    rng = np.random.default_rng(10 + B * R)
    K = 14
    sets, pool = _random_sets(rng, K, 20, 120, shared_pool=60, shared_per_set=15)
    del sets[K - 1]  # one ID never inserted
    sets[K - 2] = set()  # one set inserted with no terms
    o = _build(oracle_mod, sets, K, B, R, 1 << 24, 2, 7)  # BF false positives ~1e-9
    phi = o.phi
    members = [x for S in sets.values() for x in S]
    fresh = [int(v) for v in rng.integers(0, 1 << 62, 40, dtype=np.uint64)]
    queries = [[x] for x in rng.choice(members, 80)] + [[x] for x in pool[:30]] + [[x] for x in fresh]
    queries += [list(rng.choice(members, 2)) for _ in range(40)] + [list(rng.choice(pool, 3)) for _ in range(40)]
    for Q in queries:
        Q = [int(x) for x in Q]
        got = list(o.query_keys(np.array(Q, np.uint64)))
        want = exact_cell_rambo(sets, phi, R, Q)
        assert got == want, Q
        truth = exact_msmt(sets, Q)
        assert set(truth) <= set(got)  # no false negatives (Sec. 4.1)
        assert K - 1 not in got  # an ID never inserted is never reported


def test_no_false_negatives_with_crowded_filters(oracle_mod):
    rng = np.random.default_rng(11)
    K, B, R = 40, 6, 3
    sets, pool = _random_sets(rng, K, 100, 400, shared_pool=200, shared_per_set=30)
    o = _build(oracle_mod, sets, K, B, R, 1 << 10, 2, 3)  # heavily loaded filters
    members = [x for S in sets.values() for x in S]
    for x in rng.choice(members, 300):
        got = set(o.query_keys(np.array([x], np.uint64)))
        assert set(exact_msmt(sets, [int(x)])) <= got


def test_sequence_queries_equal_exact_cell_on_kmers(oracle_mod):
    rng = np.random.default_rng(12)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    K, B, R, k = 10, 4, 3, 31
    seqs = {i: bytes(acgt[rng.integers(0, 4, int(rng.integers(40, 400)))]) for i in range(K)}
    o = oracle_mod.Oracle(K, B, R, 1 << 24, 2, 5)
    for i, s in seqs.items():
        o.insert_seq(i, s, k)
    kset = {i: {int(v) for v in oracle_mod.kmers(s, k)} for i, s in seqs.items()}
    for _ in range(60):
        i = int(rng.integers(0, K))
        s = seqs[i]
        a = int(rng.integers(0, len(s) - k))
        b = int(rng.integers(a + k, len(s) + 1))
        q = s[a:b]
        Q = [int(v) for v in oracle_mod.kmers(q, k)]
        assert list(o.query_seq(q, k)) == exact_cell_rambo(kset, o.phi, R, Q)
        assert i in o.query_seq(q, k)


# --------------------------------------------------------------------------
# special cases that reduce to a textbook Bloom filter
# --------------------------------------------------------------------------

def test_single_cell_is_one_bloom_filter(oracle_mod):
    # B=1, R=1: the structure is a single Bloom filter of the union of all
    # sets; the answer is every registered set when the filter says yes.
    rng = np.random.default_rng(13)
    K, m, eta = 9, 1 << 9, 3
    sets, _ = _random_sets(rng, K, 10, 40)
    del sets[4]
    o = _build(oracle_mod, sets, K, 1, 1, m, eta, 17)
    bits = np.zeros(m, bool)
    for S in sets.values():
        for x in S:
            for j in range(eta):
                bits[o.pos(0, j, x)] = True  # textbook insert (Sec. 2)
    assert np.array_equal(o.bf_bits(0, 0).astype(bool), bits)
    regd = sorted(sets)
    for x in [int(v) for v in rng.integers(0, 1 << 62, 300, dtype=np.uint64)] + list(sets[0]):
        yes = all(bits[o.pos(0, j, x)] for j in range(eta))  # textbook query (Sec. 2)
        assert list(o.query_keys(np.array([x], np.uint64))) == (regd if yes else [])


def test_one_table_returns_members_of_hit_cells(oracle_mod):
    rng = np.random.default_rng(14)
    K, B = 30, 5
    sets, _ = _random_sets(rng, K, 30, 60)
    o = _build(oracle_mod, sets, K, B, 1, 1 << 11, 2, 19)
    for x in [int(v) for v in rng.integers(0, 1 << 62, 200, dtype=np.uint64)] + list(sets[3])[:20]:
        hit = {b for b in range(B) if o.bf_contains(0, b, x)}
        want = sorted(i for i in sets if o.phi(0, i) in hit)
        assert list(o.query_keys(np.array([x], np.uint64))) == want


# --------------------------------------------------------------------------
# identities of Algorithm 2
# --------------------------------------------------------------------------

def test_conjunction_equals_intersection_of_single_term_answers(oracle_mod):
    # Sec. 3.2.1: the answer for Q is the conjunction of the per-term answers;
    # because each table partitions the sets this holds exactly, also with
    # Bloom-filter false positives present.
    rng = np.random.default_rng(15)
    K, B, R = 50, 6, 3
    sets, pool = _random_sets(rng, K, 100, 300, shared_pool=100, shared_per_set=40)
    o = _build(oracle_mod, sets, K, B, R, 1 << 11, 2, 23)  # plenty of false positives
    for _ in range(100):
        Q = [int(x) for x in rng.choice(pool, int(rng.integers(2, 6)))]
        if rng.random() < 0.3:
            Q.append(int(rng.integers(0, 1 << 62)))
        want = set(range(K))
        for x in Q:
            want &= set(o.query_keys(np.array([x], np.uint64)))
        assert list(o.query_keys(np.array(Q, np.uint64))) == sorted(want)
    # duplicate terms change nothing
    Q = [int(x) for x in pool[:3]]
    assert list(o.query_keys(np.array(Q + Q, np.uint64))) == list(o.query_keys(np.array(Q, np.uint64)))


def test_index_bits_do_not_depend_on_insert_order_or_split(oracle_mod):
    rng = np.random.default_rng(16)
    K, B, R, m, eta = 20, 5, 3, 1 << 12, 2
    sets, _ = _random_sets(rng, K, 50, 150)
    a = _build(oracle_mod, sets, K, B, R, m, eta, 31)
    b = _build(oracle_mod, sets, K, B, R, m, eta, 31, order=list(reversed(sorted(sets))))
    c = oracle_mod.Oracle(K, B, R, m, eta, 31)
    for i in sorted(sets):  # each set inserted in two parts
        keys = np.array(sorted(sets[i]), np.uint64)
        c.insert_keys(i, keys[1::2])
        c.insert_keys(i, keys[0::2])
    ids = np.array(sorted(sets), np.uint64)
    keys = np.concatenate([np.array(sorted(sets[i]), np.uint64) for i in sorted(sets)])
    off = np.zeros(len(sets) + 1, np.uint64)
    np.cumsum([len(sets[i]) for i in sorted(sets)], out=off[1:])
    d = oracle_mod.Oracle(K, B, R, m, eta, 31)
    d.insert_keys_batch(ids, keys, off, nthreads=4)
    for r in range(R):
        for cell in range(B):
            ref = a.export_bf(r, cell)
            for other in (b, c, d):
                assert np.array_equal(ref, other.export_bf(r, cell))


def test_batch_sequence_insert_equals_one_by_one(oracle_mod):
    rng = np.random.default_rng(17)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    K, B, R, m, eta, k = 12, 4, 3, 1 << 14, 2, 31
    lens = rng.integers(0, 300, K)
    lens[2] = 30  # shorter than k: registered, no terms
    seqs = [acgt[rng.integers(0, 4, int(n))] for n in lens]
    a = oracle_mod.Oracle(K, B, R, m, eta, 3)
    for i, s in enumerate(seqs):
        a.insert_seq(i, s, k)
    bases = np.concatenate(seqs)
    off = np.zeros(K + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    for nt in (1, 3):
        b = oracle_mod.Oracle(K, B, R, m, eta, 3)
        b.insert_seq_batch(np.arange(K, dtype=np.uint64), bases, off, k, nthreads=nt)
        for r in range(R):
            for cell in range(B):
                assert np.array_equal(a.export_bf(r, cell), b.export_bf(r, cell))
        assert np.array_equal(a.registered(), b.registered())
    assert a.registered()[2]


def test_batch_query_equals_single_queries(oracle_mod):
    rng = np.random.default_rng(18)
    K, B, R = 30, 5, 3
    sets, pool = _random_sets(rng, K, 50, 100, shared_pool=40, shared_per_set=10)
    o = _build(oracle_mod, sets, K, B, R, 1 << 12, 2, 29)
    qs = [[int(x) for x in rng.choice(pool, int(rng.integers(1, 4)))] for _ in range(50)]
    data = np.array([x for q in qs for x in q], np.uint64)
    off = np.zeros(len(qs) + 1, np.uint64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    for nt in (1, 4):
        ids, ioff = o.query_batch("keys", data, off, nthreads=nt)
        for t, q in enumerate(qs):
            assert list(ids[ioff[t]:ioff[t + 1]]) == list(o.query_keys(np.array(q, np.uint64)))


def test_errors(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(10, 4, 2, 1000, 2, 1)  # m not a power of two
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(10, 0, 2, 1024, 2, 1)
    o = oracle_mod.Oracle(10, 4, 2, 1 << 10, 2, 1)
    with pytest.raises(oracle_mod.OracleError) as e:
        o.insert_keys(10, np.array([1], np.uint64))
    assert e.value.code == oracle_mod.ERANGE
    with pytest.raises(oracle_mod.OracleError) as e:
        o.query_keys(np.zeros(0, np.uint64))
    assert e.value.code == oracle_mod.EINVAL
    with pytest.raises(oracle_mod.OracleError) as e:
        o.query_seq(b"ACGT" * 7, 31)  # 28 bases < k
    assert e.value.code == oracle_mod.EBADSEQ
    with pytest.raises(oracle_mod.OracleError) as e:
        o.query_seq(b"ACGT" * 10 + b"N", 31)
    assert e.value.code == oracle_mod.EBADSEQ


# --------------------------------------------------------------------------
# false-positive rates against the analysis (Sec. 2, Lemma 4.1, Lemma 4.2)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def fp_setup(oracle_mod):
    rng = np.random.default_rng(20)
    K, B, R, m, eta = 160, 8, 4, 1 << 17, 2
    n_per = 1500
    keys = rng.integers(0, 1 << 62, K * n_per, dtype=np.uint64)
    off = np.arange(K + 1, dtype=np.uint64) * np.uint64(n_per)
    o = oracle_mod.Oracle(K, B, R, m, eta, 77)
    o.insert_keys_batch(np.arange(K, dtype=np.uint64), keys, off, nthreads=4)
    fill = o.cell_popcount() / m
    phi = o.phi_table()  # [K, R]
    return o, rng, K, B, R, m, eta, fill, phi, keys, n_per


def test_bloom_cell_false_positive_rate(fp_setup):
    o, rng, K, B, R, m, eta, fill, phi, keys, n_per = fp_setup
    fresh = [int(v) for v in rng.integers(0, 1 << 62, 3000, dtype=np.uint64)]
    hits = np.zeros((R, B))
    for x in fresh:
        for r in range(R):
            for b in range(B):
                hits[r, b] += o.bf_contains(r, b, x)
    p = fill**eta  # chance all eta uniform positions land on set bits
    exp = len(fresh) * p.sum()
    sd = np.sqrt(len(fresh) * (p * (1 - p)).sum())
    assert abs(hits.sum() - exp) < 5 * sd
    # Sec. 2 closed form with n = keys inserted in the cell
    n_cell = np.zeros((R, B))
    for r in range(R):
        n_cell[r] = np.bincount(phi[:, r], minlength=B) * n_per
    p_formula = (1 - (1 - 1 / m) ** (eta * n_cell)) ** eta
    assert np.allclose(p_formula, p, rtol=0.05)  # fill matches its expectation
    assert abs(hits.sum() - len(fresh) * p_formula.sum()) < 5 * sd + 0.05 * exp


def _multiplicity_run(o, rng, K, B, R, eta, fill, phi, V, n_keys):
    """Sec. 5.2's evaluation: fresh keys inserted into V random sets each, then
    queried.  Returns per-key arrays (false IDs observed, false IDs predicted
    exactly given the partition and cell fills, any false ID) and p, the BFU
    false-positive rate averaged over the sets' own cells."""
    obs = np.zeros(n_keys)
    pred = np.zeros(n_keys)
    for t in range(n_keys):
        x = int(rng.integers(0, 1 << 62))
        mem = rng.choice(K, V, replace=False) if V else np.zeros(0, np.int64)
        for i in mem:
            o.insert_keys(int(i), np.array([x], np.uint64))
        got = set(int(v) for v in o.query_keys(np.array([x], np.uint64)))
        assert set(int(i) for i in mem) <= got  # no false negatives
        non = np.setdiff1d(np.arange(K), mem)
        obs[t] = len(got - set(int(i) for i in mem))
        pr = np.ones(non.size)
        for r in range(R):
            shared = np.isin(phi[non, r], phi[mem, r]) if V else np.zeros(non.size, bool)
            pr *= np.where(shared, 1.0, fill[r, phi[non, r]] ** eta)
        pred[t] = pr.sum()
    p = float(np.mean([fill[r, phi[:, r]] ** eta for r in range(R)]))
    return obs, pred, p


@pytest.mark.parametrize("V", [0, 1, 3, 8])
def test_rambo_false_positive_rate_lemma_4_1(fp_setup, V):
    o, rng, K, B, R, m, eta, fill, phi, keys, n_per = fp_setup
    n_keys = 1500
    obs, pred, p = _multiplicity_run(o, rng, K, B, R, eta, fill, phi, V, n_keys)
    n_non = K - V
    se = max(obs.std(), 1.0) / np.sqrt(n_keys)  # standard error of the mean false-ID count
    # exact conditional prediction given the partition and the cell fills
    assert abs(obs.mean() - pred.mean()) < 4 * se + 0.05 * pred.mean()
    # Lemma 4.1: F_p = (p (1-1/B)^V + 1 - (1-1/B)^V)^R per non-member set; it
    # averages over the partition's randomness, which one instance only samples,
    # hence the 15% slack on top of the sampling error
    q = (1 - 1 / B) ** V
    Fp = (p * q + 1 - q) ** R
    assert abs(obs.mean() / n_non - Fp) < 4 * se / n_non + 0.15 * Fp
    # Lemma 4.2: P(any wrong ID) <= K (1 - (1-p)(1-1/B)^V)^R
    delta = K * (1 - (1 - p) * q) ** R
    any_fp = (obs > 0).mean()
    assert any_fp <= min(1.0, delta) + 4 * np.sqrt(max(any_fp, 1 / n_keys) / n_keys)


def test_folding_over_equals_half_the_cells(oracle_mod):
    # appendix, folding over: OR-ing cell b + B/2 onto cell b gives the Bloom
    # filter of the union of both cells' sets, i.e. the structure built with
    # B/2 cells; the partition hash mod B then mod B/2 is the hash mod B/2.
    rng = np.random.default_rng(30)
    K, B, R, m = 40, 12, 3, 1 << 12
    sets, _ = _random_sets(rng, K, 30, 80)
    full = _build(oracle_mod, sets, K, B, R, m, 2, 99)
    half = _build(oracle_mod, sets, K, B // 2, R, m, 2, 99)
    for r in range(R):
        for b in range(B // 2):
            assert np.array_equal(full.export_bf(r, b) | full.export_bf(r, b + B // 2), half.export_bf(r, b))
        for i in range(K):
            assert full.phi(r, i) % (B // 2) == half.phi(r, i)


# --------------------------------------------------------------------------
# two-level hash and merge (Sec. 5.2, appendix)
# --------------------------------------------------------------------------

def test_two_level_hash_routes_sets_to_node_ranges(oracle_mod):
    K, Bl, nodes, R = 3000, 8, 6, 4
    o = oracle_mod.Oracle(K, Bl, R, 1 << 8, 2, 5, nodes=nodes, tau_seed=77)
    plain = oracle_mod.Oracle(K, Bl, R, 1 << 8, 2, 5)
    for i in range(0, K, 7):
        t = o.node(i)
        assert 0 <= t < nodes
        for r in range(R):
            cell = o.phi(r, i)
            # B_local * tau(i) + phi_r(i), phi_r being the plain partition over B_local cells
            assert cell == Bl * t + plain.phi(r, i)
    # one node: the plain partition
    one = oracle_mod.Oracle(K, Bl, R, 1 << 8, 2, 5, nodes=1, tau_seed=77)
    assert np.array_equal(one.phi_table(), plain.phi_table())


def test_two_level_hash_collision_rate_is_one_over_total_cells(oracle_mod):
    # appendix: the combined mapping collides two sets with probability 1/B, B = b * nodes
    K, Bl, nodes, R = 6000, 10, 5, 3
    o = oracle_mod.Oracle(K, Bl, R, 1 << 8, 2, 11, nodes=nodes, tau_seed=3)
    tab = o.phi_table()
    rng = np.random.default_rng(5)
    i = rng.integers(0, K, 40000)
    j = rng.integers(0, K, 40000)
    keep = i != j
    B = Bl * nodes
    coll = (tab[i[keep]] == tab[j[keep]]).mean(axis=0)
    sd = np.sqrt((1 / B) * (1 - 1 / B) / keep.sum())
    assert np.all(np.abs(coll - 1 / B) < 5 * sd + 0.002)


def test_node_local_structures_merge_into_the_stacked_one(oracle_mod):
    rng = np.random.default_rng(31)
    K, Bl, nodes, R, m = 60, 4, 3, 3, 1 << 11
    sets, _ = _random_sets(rng, K, 20, 80)
    whole = oracle_mod.Oracle(K, Bl, R, m, 2, 9, nodes=nodes, tau_seed=4)
    for i in sorted(sets):
        whole.insert_keys(i, np.array(sorted(sets[i]), np.uint64))
    parts = [oracle_mod.Oracle(K, Bl, R, m, 2, 9, nodes=nodes, tau_seed=4) for _ in range(nodes)]
    for i in sorted(sets):
        parts[whole.node(i)].insert_keys(i, np.array(sorted(sets[i]), np.uint64))
    for t in range(nodes):  # a node only touches its own cell range
        for r in range(R):
            for b in range(Bl * nodes):
                if not (Bl * t <= b < Bl * (t + 1)):
                    assert not parts[t].export_bf(r, b).any()
    merged = parts[0]
    for t in range(1, nodes):
        merged.merge(parts[t])
    for r in range(R):
        for b in range(Bl * nodes):
            assert np.array_equal(merged.export_bf(r, b), whole.export_bf(r, b))
    assert np.array_equal(merged.registered(), whole.registered())
    # folding the stacked structure: OR of the halves, cells taken mod B/2
    before = {(r, b): whole.export_bf(r, b) for r in range(R) for b in range(Bl * nodes)}
    phi_before = whole.phi_table()
    whole.fold()
    half = Bl * nodes // 2
    for r in range(R):
        for b in range(half):
            assert np.array_equal(whole.export_bf(r, b), before[(r, b)] | before[(r, b + half)])
    assert np.array_equal(whole.phi_table(), phi_before % half)
