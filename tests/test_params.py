"""The parameter chooser (Sec. 5.1 "Parameter Selection"; Lemmas 4.2 and 4.4,
Theorem 4.3), pinned to things other than its own formulas:

- Lemma 4.2 worked by hand on small numbers, and the smallest such R;
- Lemma 4.4's expected query time scanned numerically over B, whose minimum
  must sit where the chooser puts B;
- the failure probability of a structure built with the chosen parameters,
  measured by brute force on the CPU oracle, against the target delta;
- the Bloom-filter sizing, through the false-positive rate the oracle's
  filters actually show when filled as the chooser assumed;
- the sampled mean set size (Sec. 5.1: measured on the first sets of the
  stream), against distinct counts taken here with Python sets.

Host-only: the chooser involves no GPU."""
import math

import numpy as np
import pytest

import synth


def test_lemma_4_2_worked_by_hand():
    from paper_1910_02611_gb300 import suggest_params

    # p = 0.25 gives eta0 = log2(1/p) = 2, so Lemma 4.4 puts B at
    # sqrt(K V / eta) = sqrt(100 * 2 / 2) = 10.  Lemma 4.2 with B = 10, V = 2:
    #   f = 1 - (1 - 0.25) * (1 - 1/10)^2 = 1 - 0.75 * 0.81 = 0.3925
    #   K f^7 = 100 * 0.3925^7 = 0.1435... > 0.1
    #   K f^8 = 100 * 0.3925^8 = 0.0563... <= 0.1   -> R = 8
    got = suggest_params(100, 1000.0, V=2.0, p=0.25, delta=0.1)
    assert got["B"] == 10 and got["R"] == 8
    # delta = 0.2: 0.1435 <= 0.2 already at R = 7; R = 6 gives 0.3657 > 0.2
    assert suggest_params(100, 1000.0, V=2.0, p=0.25, delta=0.2)["R"] == 7
    # V = 1 (keys in one set): B = round(sqrt(100 * 1 / 2)) = 7, so
    # f = 1 - 0.75 * (6/7) = 0.357142...; 100 f^6 = 0.2075 > 0.1, 100 f^7 = 0.0741 <= 0.1
    got = suggest_params(100, 1000.0, V=1.0, p=0.25, delta=0.1)
    assert got["B"] == 7 and got["R"] == 7


@pytest.mark.parametrize("K,V,p", [(2000, 2.0, 0.01), (10**5, 20.0, 0.01), (500, 1.0, 0.25), (10**4, 4.0, 0.05)])
def test_b_minimises_lemma_4_4_expected_query_time(K, V, p):
    from paper_1910_02611_gb300 import suggest_params

    got = suggest_params(K, 1000.0, V=V, p=p, delta=0.5)
    eta = min(max(math.log2(1 / p), 1.0), 4.0)  # the Bloom-filter optimum eta the chooser sizes B with
    R = got["R"]
    Bs = np.arange(1, 4097, dtype=np.float64)
    cost = Bs * R * eta + (K / Bs) * (V + Bs * p) * R  # Lemma 4.4, evaluated at every B
    b_best = int(Bs[np.argmin(cost)])
    assert abs(got["B"] - b_best) <= 1
    # and the chooser's B costs within a hair of the best
    assert cost[got["B"] - 1] <= cost[b_best - 1] * 1.001


def test_failure_rate_of_the_chosen_structure_is_within_delta(oracle_mod):
    # Lemma 4.2 bounds P(any wrong ID for a query) by delta; build the chosen
    # structure in the oracle and count, over many fresh queries whose key is
    # in exactly V sets, how often the answer holds an ID it should not
    from paper_1910_02611_gb300 import suggest_params

    rng = np.random.default_rng(11)
    K, V, n_set, p, delta = 64, 2, 200, 0.2, 0.3
    got = suggest_params(K, float(n_set), V=float(V), p=p, delta=delta)
    B, R, m, eta = got["B"], got["R"], got["m"], got["eta"]
    o = oracle_mod.Oracle(K, B, R, m, eta, 5)
    for i in range(K):
        o.insert_keys(i, rng.integers(0, 1 << 62, n_set, dtype=np.uint64))
    trials, wrong = 3000, 0
    for _ in range(trials):
        x = int(rng.integers(0, 1 << 62))
        owners = {int(i) for i in rng.choice(K, V, replace=False)}  # x is in exactly V sets
        ans = _answer_with_key_in(o, x, owners, K, B, R)
        wrong += bool(ans - owners)  # no false negatives; any other ID is wrong
    rate = wrong / trials
    sd = math.sqrt(delta * (1 - delta) / trials)
    assert rate <= delta + 4 * sd, (rate, delta, got)


def _answer_with_key_in(o, x, owners, K, B, R):
    """Algorithm 2's answer for key x had x been inserted into the owner sets
    of structure o: inserting x only sets bits in the owners' cells, so in
    table r the hit cells are those cells plus every other cell whose filter
    already holds x; the answer is the per-table union of the hit cells' sets,
    intersected across tables."""
    phi = _PHI_CACHE.setdefault(id(o), o.phi_table())
    ans = None
    for r in range(R):
        own_cells = {int(phi[i, r]) for i in owners}
        hit = set(own_cells)
        for b in range(B):
            if b not in hit and o.bf_contains(r, b, x):
                hit.add(b)
        g = {i for i in range(K) if int(phi[i, r]) in hit}
        ans = g if ans is None else ans & g
    return ans


_PHI_CACHE: dict = {}


def test_filters_sized_by_the_chooser_meet_the_target_rate(oracle_mod):
    # the chooser sizes each BFU for n_mean * K / B keys at rate p; filled that
    # way, the oracle's filters must show a false-positive rate of at most p
    # (m is rounded up to a power of two, so typically below)
    from paper_1910_02611_gb300 import suggest_params

    rng = np.random.default_rng(3)
    K, n_mean, p = 40, 300, 0.05
    got = suggest_params(K, float(n_mean), V=1.0, p=p, delta=0.5)
    B, m, eta = got["B"], got["m"], got["eta"]
    o = oracle_mod.Oracle(K, B, 1, m, eta, 8)
    for i in range(K):
        o.insert_keys(i, rng.integers(0, 1 << 62, n_mean, dtype=np.uint64))
    probes = rng.integers(0, 1 << 62, 4000, dtype=np.uint64)
    fp = np.mean([o.bf_contains(0, b, int(x)) for b in range(B) for x in probes[:400]])
    assert fp <= p * 1.15, (fp, got)
    # eta is the Bloom-filter optimum for the resulting load: ln 2 * m / n, rounded
    n = n_mean * K / B
    assert eta == min(max(round(math.log(2) * m / n), 1), 4)


def test_sampled_mean_set_size_counts_distinct_keys():
    from paper_1910_02611_gb300 import suggest_params, suggest_params_from_sample

    rng = np.random.default_rng(21)
    sets = [rng.integers(0, 500, int(rng.integers(1, 400)), dtype=np.uint64) for _ in range(30)]  # with repeats
    off = np.zeros(31, np.uint64)
    np.cumsum([s.size for s in sets], out=off[1:])
    data = np.concatenate(sets)
    want = float(np.mean([len(set(s.tolist())) for s in sets[:12]]))
    got = suggest_params_from_sample(1000, data, off[:13], kind="keys", V=2.0, p=0.01, delta=0.01)
    assert got["n_mean"] == pytest.approx(want, rel=1e-12)
    ref = suggest_params(1000, want, V=2.0, p=0.01, delta=0.01)
    assert {k: got[k] for k in ref} == ref


@pytest.mark.parametrize("k", [31, 31 | 0x100, 15 | 0x200, 31 | 0x300])
def test_sampled_mean_set_size_counts_distinct_kmers(oracle_mod, k):
    from paper_1910_02611_gb300 import suggest_params_from_sample

    w = synth.make("genome", 0.005, m=1 << 12)
    data = w.sets.data.copy()
    if k & 0x200:
        data[::97] = ord("N")
    n = 6
    want = float(np.mean([len(set(oracle_mod.kmers(data[int(w.sets.offsets[t]):int(w.sets.offsets[t + 1])], k).tolist()))
                          for t in range(n)]))
    got = suggest_params_from_sample(w.K, data, w.sets.offsets[: n + 1], kind="seq", k=k, V=1.0, p=0.05, delta=0.5)
    assert got["n_mean"] == pytest.approx(want, rel=1e-12)


def test_unreachable_failure_rate_reports_erange():
    from paper_1910_02611_gb300 import ERANGE, RamboError, suggest_params

    with pytest.raises(RamboError) as e:
        suggest_params(10**6, 1000, V=500.0, p=0.2, delta=1e-9)
    assert e.value.code == ERANGE and e.value.params["R"] == 16  # RAMBO_MAX_R


def test_sample_errors():
    from paper_1910_02611_gb300 import EBADSEQ, EINVAL, RamboError, suggest_params_from_sample

    with pytest.raises(RamboError) as e:
        suggest_params_from_sample(10, np.frombuffer(b"ACGTNACGT" * 5, np.uint8), np.array([0, 45], np.uint64),
                                   kind="seq", k=31)
    assert e.value.code == EBADSEQ
    with pytest.raises(RamboError) as e:  # a sample with no key at all
        suggest_params_from_sample(10, np.frombuffer(b"ACGT", np.uint8), np.array([0, 4], np.uint64), kind="seq", k=31)
    assert e.value.code == EINVAL
