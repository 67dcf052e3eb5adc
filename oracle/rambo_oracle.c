/*
 * rambo_oracle.c -- a plain, slow, obviously correct CPU RAMBO.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  The GPU
 * library shares no code, header, table or helper with it; both are written
 * independently from the same written hash/layout specification, restated
 * below.
 *
 * What it computes (RAMBO, Gupta et al., arXiv 1910.02611):
 *   - Bloom filter (Sec. 2 "Preliminaries"): an m-bit array; inserting a key
 *     sets the eta bits h_1(x)..h_eta(x); a key is "in" the filter iff all eta
 *     bits are set.
 *   - RAMBO (Sec. 3): R tables of B cells; each cell is a Bloom filter of the
 *     union (BFU) of the sets that the table's partition hash phi_r sends to it.
 *     Here each of the B*R BFUs is its own separate m-bit array (the paper's
 *     picture), NOT the bit-sliced layout the GPU library uses.
 *   - Insertion: Algorithm 1 (Sec. 3.1), with phi applied to the SET identity
 *     (Sec. 3.1 text and Fig. 1 caption; the algorithm box writes phi_d(x),
 *     read as phi_d(S_i)).
 *   - Query: Algorithm 2 (Sec. 3.2): per table r, G_r = union of SetIDs(M[b,r])
 *     over the cells b whose BF contains every term of Q, testing the terms in
 *     order and stopping at the first one that is absent (Sec. 3.2.1: the first
 *     FALSE is conclusive); A = intersection of the G_r, reported ascending.
 *     SetIDs(M[b,r]) is the set of *inserted* (registered) set IDs i with
 *     phi_r(i) = b.
 *   - Large sequence query (Sec. 3.2.1): Q = every length-k window of the
 *     sequence (k = 31 for genomes, Sec. 5.2).
 *
 * Hash / encoding specification (the paper only says "universal" and
 * "2-universal"; these are this project's concrete choices):
 *   SplitMix64 (Steele, Lea, Flood, OOPSLA 2014):
 *     next(s): s += 0x9E3779B97F4A7C15; return mix64(s)
 *     mix64(z): z = (z ^ (z>>30)) * 0xBF58476D1CE4E5B9;
 *               z = (z ^ (z>>27)) * 0x94D049BB133111EB;  return z ^ (z>>31)
 *   Parameters from one seed (state starts at seed), drawn in this order:
 *     for r in [0,R): a_r = 1 + next() mod (P-1);  c_r = next() mod P
 *     for r in [0,R): for j in [0,eta): s_{r,j} = next() | 1
 *     with P = 2^61 - 1.
 *   Partition hash (Carter-Wegman, 2-universal), set ID i:
 *     phi_r(i) = ((a_r * i + c_r) mod P) mod B
 *   Bloom-filter position (multiply-shift, Dietzfelbinger et al. 1997), m = 2^L:
 *     h_{r,j}(x) = (s_{r,j} * mix64(x) mod 2^64) >> (64 - L)
 *     The eta positions are shared by the B cells of one table and differ
 *     between tables.
 *   k-mer key: bases A/a=0, C/c=1, G/g=2, T/t=3; the window starting at p is
 *     sum_{t<k} code(seq[p+t]) * 4^(k-1-t) (first base most significant),
 *     1 <= k <= 32.  Any other byte is an error, unless the k argument
 *     carries ORC_SKIPN: then every window holding such a byte is skipped
 *     and a query sequence with no other window is an error.
 *
 * Parity pins: tests/test_oracle_*.py (SplitMix64 published outputs, big-int
 * arithmetic for phi, closed forms for k-mers, brute-force exact MSMT on tiny
 * inputs, Bloom/RAMBO false-positive statistics against Sec. 2 and Lemma 4.1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ERANGE (-2)
#define ORC_EBADSEQ (-3)
#define ORC_ENOMEM (-4)

static const uint64_t ORC_P = (1ULL << 61) - 1;

typedef struct orc {
    uint64_t K;          /* set-ID capacity: IDs are 0..K-1 */
    uint32_t B, R, eta, L;
    uint64_t m;          /* bits per Bloom filter, 2^L */
    uint64_t seed;
    uint64_t *a, *c;     /* phi parameters, R each */
    uint32_t B_local;    /* cells per node (two-level hash); B_local = B with one node */
    uint32_t n_nodes;    /* nodes of the two-level hash (1 = plain partition) */
    uint64_t a_tau, c_tau; /* node hash tau(i) = ((a_tau i + c_tau) mod P) mod n_nodes */
    uint64_t *s;         /* position multipliers, R*eta */
    uint64_t wpb;        /* 64-bit words per Bloom filter */
    uint64_t *bits;      /* BF of (table r, cell b) at bits + (r*B + b)*wpb */
    uint64_t *reg;       /* registered-set bitmap, K bits */
    uint64_t *mem_off;   /* R*B+1 offsets into mem_ids */
    uint32_t *mem_ids;   /* for each (r,b): the IDs i < K with phi_r(i)=b, ascending */
} orc_t;

/* ---------------- hash primitives ---------------- */

uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t *state) {
    *state += 0x9E3779B97F4A7C15ULL;
    return orc_mix64(*state);
}

/* Cell of set i in table r.  Plain: phi_r(i) = ((a_r i + c_r) mod P) mod B.
 * Two-level (Sec. 5.2, appendix): B_local * tau(i) + phi_r(i) with phi_r over
 * B_local cells and tau over the nodes.  After folding over (B halved f
 * times) the cell is the original cell mod the current B. */
uint32_t orc_phi(const orc_t *o, uint32_t r, uint64_t set_id) {
    unsigned __int128 v = (unsigned __int128)o->a[r] * set_id + o->c[r];
    uint64_t local = (uint64_t)(v % ORC_P) % o->B_local;
    uint64_t node = 0;
    if (o->n_nodes > 1) {
        unsigned __int128 t = (unsigned __int128)o->a_tau * set_id + o->c_tau;
        node = (uint64_t)(t % ORC_P) % o->n_nodes;
    }
    return (uint32_t)((o->B_local * node + local) % o->B);
}

uint64_t orc_pos(const orc_t *o, uint32_t r, uint32_t j, uint64_t key) {
    uint64_t prod = o->s[(uint64_t)r * o->eta + j] * orc_mix64(key);
    return prod >> (64 - o->L);
}

int orc_base_code(uint8_t ch) {
    switch (ch) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/* k may carry ORC_CANONICAL: each window's key is then the smaller of the
 * window and its reverse complement (the same DNA read on the other strand:
 * bases in reverse order, A<->T and C<->G, i.e. code c -> 3 - c). */
#define ORC_CANONICAL 0x100u
/* k may carry ORC_SKIPN: a byte outside ACGTacgt (an unresolved base such as
 * N) no longer rejects the sequence; every window that holds one is left
 * out, and the sequence's terms are its other windows (Sec. 3.2.1's sliding
 * window over the resolved stretches of the read). */
#define ORC_SKIPN 0x200u
#define ORC_KFLAGS (0xffu | ORC_CANONICAL | ORC_SKIPN)

/* 1 when the k bytes seq[p .. p+k) are all in ACGTacgt. */
static int window_valid(const uint8_t *seq, uint64_t p, uint32_t k) {
    for (uint32_t t = 0; t < k; ++t)
        if (orc_base_code(seq[p + t]) < 0) return 0;
    return 1;
}

/* Key of the window seq[p .. p+k): forward, or canonical. */
static uint64_t window_key(const uint8_t *seq, uint64_t p, uint32_t k, int canon) {
    uint64_t fwd = 0, rc = 0;
    for (uint32_t t = 0; t < k; ++t) fwd = fwd * 4 + (uint64_t)orc_base_code(seq[p + t]);
    if (!canon) return fwd;
    for (uint32_t t = 0; t < k; ++t) rc = rc * 4 + (uint64_t)(3 - orc_base_code(seq[p + k - 1 - t]));
    return rc < fwd ? rc : fwd;
}

/* Writes the window keys of seq into out (if out != NULL), in window order.
 * Returns the number of windows: n-k+1 (0 when n < k), or with ORC_SKIPN the
 * number of windows free of bytes outside ACGTacgt.  Without ORC_SKIPN such
 * a byte anywhere gives ORC_EBADSEQ.  ORC_EINVAL for k outside [1,32] (or
 * unknown flag bits). */
int64_t orc_kmers(const uint8_t *seq, uint64_t n, uint32_t kflags, uint64_t *out) {
    const uint32_t k = kflags & 0xffu;
    const int canon = (kflags & ORC_CANONICAL) != 0;
    const int skipn = (kflags & ORC_SKIPN) != 0;
    if (k < 1 || k > 32 || (kflags & ~ORC_KFLAGS)) return ORC_EINVAL;
    if (!skipn)
        for (uint64_t p = 0; p < n; ++p)
            if (orc_base_code(seq[p]) < 0) return ORC_EBADSEQ;
    if (n < k) return 0;
    uint64_t nw = 0;
    for (uint64_t p = 0; p + k <= n; ++p) {
        if (skipn && !window_valid(seq, p, k)) continue;
        if (out) out[nw] = window_key(seq, p, k, canon);
        ++nw;
    }
    return (int64_t)nw;
}

/* ---------------- construction of the structure ---------------- */

void orc_destroy(orc_t *o) {
    if (!o) return;
    free(o->a); free(o->c); free(o->s);
    free(o->bits); free(o->reg); free(o->mem_off); free(o->mem_ids);
    free(o);
}

/* Parameters as in the specification above.  Returns NULL on bad parameters
 * (B=0, R=0, eta=0, K=0, K > 2^32, m not a power of two in [2, 2^32]) or when
 * memory runs out. */
static int build_members(orc_t *o);

static orc_t *create_impl(uint64_t K, uint32_t B_local, uint32_t n_nodes, uint32_t R, uint64_t m,
                          uint32_t eta, uint64_t seed, uint64_t tau_seed) {
    uint64_t Bfull = (uint64_t)B_local * n_nodes;
    if (K == 0 || K > (1ULL << 32) || B_local == 0 || n_nodes == 0 || Bfull > 65535 || R == 0 || R > 64 ||
        eta == 0 || eta > 64 || m < 2 || m > (1ULL << 32) || (m & (m - 1)))
        return NULL;
    uint32_t B = (uint32_t)Bfull;
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    o->K = K; o->B = B; o->R = R; o->eta = eta; o->m = m; o->seed = seed;
    o->B_local = B_local; o->n_nodes = n_nodes;
    if (n_nodes > 1) {
        uint64_t ts = tau_seed;
        o->a_tau = 1 + orc_splitmix64_next(&ts) % (ORC_P - 1);
        o->c_tau = orc_splitmix64_next(&ts) % ORC_P;
    }
    uint32_t L = 0;
    while ((1ULL << L) < m) ++L;
    o->L = L;
    o->a = (uint64_t *)malloc(sizeof(uint64_t) * R);
    o->c = (uint64_t *)malloc(sizeof(uint64_t) * R);
    o->s = (uint64_t *)malloc(sizeof(uint64_t) * R * eta);
    o->wpb = (m + 63) / 64;
    o->bits = (uint64_t *)calloc((size_t)R * B * o->wpb, sizeof(uint64_t));
    o->reg = (uint64_t *)calloc((K + 63) / 64, sizeof(uint64_t));
    o->mem_off = (uint64_t *)calloc((size_t)R * B + 1, sizeof(uint64_t));
    o->mem_ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)R * K);
    if (!o->a || !o->c || !o->s || !o->bits || !o->reg || !o->mem_off || !o->mem_ids) {
        orc_destroy(o);
        return NULL;
    }
    uint64_t st = seed;
    for (uint32_t r = 0; r < R; ++r) {
        o->a[r] = 1 + orc_splitmix64_next(&st) % (ORC_P - 1);
        o->c[r] = orc_splitmix64_next(&st) % ORC_P;
    }
    for (uint32_t r = 0; r < R; ++r)
        for (uint32_t j = 0; j < eta; ++j)
            o->s[(uint64_t)r * eta + j] = orc_splitmix64_next(&st) | 1ULL;
    if (build_members(o)) { orc_destroy(o); return NULL; }
    return o;
}

/* SetIDs(M[b,r]) over the whole ID range, ascending: counting sort by cell. */
static int build_members(orc_t *o) {
    const uint32_t R = o->R, B = o->B;
    const uint64_t K = o->K;
    memset(o->mem_off, 0, sizeof(uint64_t) * ((size_t)R * B + 1));
    for (uint32_t r = 0; r < R; ++r)
        for (uint64_t i = 0; i < K; ++i)
            o->mem_off[(uint64_t)r * B + orc_phi(o, r, i) + 1] += 1;
    for (uint64_t t = 0; t < (uint64_t)R * B; ++t) o->mem_off[t + 1] += o->mem_off[t];
    uint64_t *fill = (uint64_t *)calloc((size_t)R * B, sizeof(uint64_t));
    if (!fill) return ORC_ENOMEM;
    for (uint32_t r = 0; r < R; ++r)
        for (uint64_t i = 0; i < K; ++i) {
            uint64_t cell = (uint64_t)r * B + orc_phi(o, r, i);
            o->mem_ids[o->mem_off[cell] + fill[cell]++] = (uint32_t)i;
        }
    free(fill);
    return ORC_OK;
}

orc_t *orc_create(uint64_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint64_t seed) {
    return create_impl(K, B, 1, R, m, eta, seed, 0);
}

/* Two-level hash (Sec. 5.2, appendix): n_nodes node-local structures of
 * B_local cells stacked into one of B_local * n_nodes cells; set i lives in
 * cell B_local * tau(i) + phi_r(i) of table r.  tau's parameters come from
 * SplitMix64 started at tau_seed: a = 1 + next() mod (P-1), c = next() mod P. */
orc_t *orc_create_stacked(uint64_t K, uint32_t B_local, uint32_t n_nodes, uint32_t R, uint64_t m, uint32_t eta,
                          uint64_t seed, uint64_t tau_seed) {
    return create_impl(K, B_local, n_nodes, R, m, eta, seed, tau_seed);
}

uint32_t orc_node(const orc_t *o, uint64_t set_id) {
    if (o->n_nodes <= 1) return 0;
    unsigned __int128 t = (unsigned __int128)o->a_tau * set_id + o->c_tau;
    return (uint32_t)((uint64_t)(t % ORC_P) % o->n_nodes);
}

uint64_t orc_param_a(const orc_t *o, uint32_t r) { return o->a[r]; }
uint64_t orc_param_c(const orc_t *o, uint32_t r) { return o->c[r]; }
uint64_t orc_param_s(const orc_t *o, uint32_t r, uint32_t j) { return o->s[(uint64_t)r * o->eta + j]; }

/* ---------------- Bloom filter primitives (Sec. 2) ---------------- */

static uint64_t *bf_of(const orc_t *o, uint32_t r, uint32_t b) {
    return o->bits + ((uint64_t)r * o->B + b) * o->wpb;
}

static void bf_insert(const orc_t *o, uint32_t r, uint32_t b, uint64_t x) {
    uint64_t *bf = bf_of(o, r, b);
    for (uint32_t j = 0; j < o->eta; ++j) {
        uint64_t p = orc_pos(o, r, j, x);
        bf[p >> 6] |= 1ULL << (p & 63);
    }
}

static int bf_contains(const orc_t *o, uint32_t r, uint32_t b, uint64_t x) {
    const uint64_t *bf = bf_of(o, r, b);
    for (uint32_t j = 0; j < o->eta; ++j) {
        uint64_t p = orc_pos(o, r, j, x);
        if (!((bf[p >> 6] >> (p & 63)) & 1ULL)) return 0;
    }
    return 1;
}

int orc_bf_contains(const orc_t *o, uint32_t r, uint32_t b, uint64_t x) {
    return bf_contains(o, r, b, x);
}

/* ---------------- Algorithm 1: insertion ---------------- */

static void reg_set(orc_t *o, uint64_t i) { o->reg[i >> 6] |= 1ULL << (i & 63); }
static int reg_get(const orc_t *o, uint64_t i) { return (int)((o->reg[i >> 6] >> (i & 63)) & 1ULL); }

int orc_is_registered(const orc_t *o, uint64_t i) { return i < o->K ? reg_get(o, i) : 0; }

/* Insert the terms of set S_i (a list of keys).  The set counts as inserted
 * (registered) even when it has no terms. */
int orc_insert_keys(orc_t *o, uint64_t set_id, const uint64_t *keys, uint64_t n) {
    if (set_id >= o->K) return ORC_ERANGE;
    reg_set(o, set_id);
    for (uint64_t t = 0; t < n; ++t)
        for (uint32_t d = 0; d < o->R; ++d)
            bf_insert(o, d, orc_phi(o, d, set_id), keys[t]);
    return ORC_OK;
}

/* Insert the k-mers of one sequence into set S_i. */
int orc_insert_seq(orc_t *o, uint64_t set_id, const uint8_t *seq, uint64_t n, uint32_t k /* may carry ORC_CANONICAL */) {
    if (set_id >= o->K) return ORC_ERANGE;
    int64_t nw = orc_kmers(seq, n, k, NULL);
    if (nw < 0) return (int)nw;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (nw > 0 ? (uint64_t)nw : 1));
    if (!keys) return ORC_ENOMEM;
    orc_kmers(seq, n, k, keys);
    int rc = orc_insert_keys(o, set_id, keys, (uint64_t)nw);
    free(keys);
    return rc;
}

/* Batch form of Algorithm 1 for many sets given as sequences (set t has ID
 * set_ids[t] and bases seq[offsets[t] .. offsets[t+1])).  With nthreads > 1,
 * thread q runs the same loops but only writes the Bloom filters of the cells
 * (r,b) with (r*B + b) mod nthreads == q; since insertion only sets bits, the
 * final bits do not depend on the order (Sec. 3.1, "conducive to updates").
 * All inputs are validated before anything is inserted. */
int orc_insert_seq_batch(orc_t *o, const uint64_t *set_ids, const uint8_t *seq,
                         const uint64_t *offsets, uint64_t n_sets, uint32_t kflags,
                         int nthreads) {
    const uint32_t k = kflags & 0xffu;
    const int canon = (kflags & ORC_CANONICAL) != 0;
    const int skipn = (kflags & ORC_SKIPN) != 0;
    if (k < 1 || k > 32 || (kflags & ~ORC_KFLAGS)) return ORC_EINVAL;
    for (uint64_t t = 0; t < n_sets; ++t) {
        if (set_ids[t] >= o->K) return ORC_ERANGE;
        if (offsets[t + 1] < offsets[t]) return ORC_EINVAL;
        int64_t nw = orc_kmers(seq + offsets[t], offsets[t + 1] - offsets[t], kflags, NULL);
        if (nw < 0) return (int)nw;
    }
    for (uint64_t t = 0; t < n_sets; ++t) reg_set(o, set_ids[t]);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        int me = 0, nt = 1;
#ifdef _OPENMP
        me = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        /* the window key, kept by dropping the oldest base and appending the
         * next; `run` counts the resolved bases ending at p (with ORC_SKIPN a
         * window is inserted only when all k of its bases are resolved) */
        uint64_t mask = k == 32 ? ~0ULL : ((1ULL << (2 * k)) - 1);
        for (uint64_t t = 0; t < n_sets; ++t) {
            const uint8_t *s = seq + offsets[t];
            uint64_t n = offsets[t + 1] - offsets[t];
            if (n < k) continue;
            for (uint32_t d = 0; d < o->R; ++d) {
                uint32_t b = orc_phi(o, d, set_ids[t]);
                if ((int)(((uint64_t)d * o->B + b) % (uint64_t)nt) != me) continue;
                uint64_t v = 0, run = 0;
                for (uint64_t p = 0; p < n; ++p) {
                    const int code = orc_base_code(s[p]);
                    run = code < 0 ? 0 : run + 1;
                    v = ((v << 2) | (uint64_t)(code < 0 ? 0 : code)) & mask;
                    if (p + 1 >= k && (!skipn || run >= k))
                        bf_insert(o, d, b, canon ? window_key(s, p + 1 - k, k, 1) : v);
                }
            }
        }
    }
    return ORC_OK;
}

/* Same as orc_insert_seq_batch for sets given as key lists. */
int orc_insert_keys_batch(orc_t *o, const uint64_t *set_ids, const uint64_t *keys,
                          const uint64_t *offsets, uint64_t n_sets, int nthreads) {
    for (uint64_t t = 0; t < n_sets; ++t) {
        if (set_ids[t] >= o->K) return ORC_ERANGE;
        if (offsets[t + 1] < offsets[t]) return ORC_EINVAL;
    }
    for (uint64_t t = 0; t < n_sets; ++t) reg_set(o, set_ids[t]);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        int me = 0, nt = 1;
#ifdef _OPENMP
        me = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        for (uint64_t t = 0; t < n_sets; ++t)
            for (uint32_t d = 0; d < o->R; ++d) {
                uint32_t b = orc_phi(o, d, set_ids[t]);
                if ((int)(((uint64_t)d * o->B + b) % (uint64_t)nt) != me) continue;
                for (uint64_t p = offsets[t]; p < offsets[t + 1]; ++p) bf_insert(o, d, b, keys[p]);
            }
    }
    return ORC_OK;
}

/* ---------------- Algorithm 2: membership query ---------------- */

typedef struct { uint64_t *G; uint64_t *A; } orc_scratch;

static int scratch_init(const orc_t *o, orc_scratch *sc) {
    uint64_t kw = (o->K + 63) / 64;
    sc->G = (uint64_t *)malloc(sizeof(uint64_t) * kw);
    sc->A = (uint64_t *)malloc(sizeof(uint64_t) * kw);
    return (sc->G && sc->A) ? ORC_OK : ORC_ENOMEM;
}
static void scratch_free(orc_scratch *sc) { free(sc->G); free(sc->A); }

/* A = intersection over r of G_r, G_r = union of SetIDs(M[b,r]) over the cells
 * b whose BF holds every term of Q.  Writes the ascending IDs (up to cap of
 * them) to out and returns how many there are. */
static int64_t query_terms(const orc_t *o, const uint64_t *Q, uint64_t nq,
                           orc_scratch *sc, uint32_t *out, uint64_t cap) {
    uint64_t kw = (o->K + 63) / 64;
    for (uint64_t w = 0; w < kw; ++w) sc->A[w] = ~0ULL;
    for (uint32_t r = 0; r < o->R; ++r) {
        memset(sc->G, 0, sizeof(uint64_t) * kw);
        for (uint32_t b = 0; b < o->B; ++b) {
            int in = 1;
            for (uint64_t t = 0; t < nq; ++t)
                if (!bf_contains(o, r, b, Q[t])) { in = 0; break; }
            if (!in) continue;
            uint64_t cell = (uint64_t)r * o->B + b;
            for (uint64_t u = o->mem_off[cell]; u < o->mem_off[cell + 1]; ++u) {
                uint32_t i = o->mem_ids[u];
                if (reg_get(o, i)) sc->G[i >> 6] |= 1ULL << (i & 63);
            }
        }
        for (uint64_t w = 0; w < kw; ++w) sc->A[w] &= sc->G[w];
    }
    int64_t cnt = 0;
    for (uint64_t i = 0; i < o->K; ++i)
        if ((sc->A[i >> 6] >> (i & 63)) & 1ULL) {
            if ((uint64_t)cnt < cap && out) out[cnt] = (uint32_t)i;
            ++cnt;
        }
    return cnt;
}

/* One query given as a list of keys (terms).  An empty list is rejected. */
int64_t orc_query_keys(const orc_t *o, const uint64_t *keys, uint64_t n,
                       uint32_t *out, uint64_t cap) {
    if (n == 0) return ORC_EINVAL;
    orc_scratch sc;
    if (scratch_init(o, &sc)) { scratch_free(&sc); return ORC_ENOMEM; }
    int64_t cnt = query_terms(o, keys, n, &sc, out, cap);
    scratch_free(&sc);
    return cnt;
}

/* One query given as a sequence: Q = its k-mers.  A sequence shorter than k
 * (no terms) or with a byte outside ACGTacgt is rejected. */
int64_t orc_query_seq(const orc_t *o, const uint8_t *seq, uint64_t n, uint32_t k,
                      uint32_t *out, uint64_t cap) {
    int64_t nw = orc_kmers(seq, n, k, NULL);
    if (nw < 0) return nw;
    if (nw == 0) return ORC_EBADSEQ;
    uint64_t *Q = (uint64_t *)malloc(sizeof(uint64_t) * (uint64_t)nw);
    if (!Q) return ORC_ENOMEM;
    orc_kmers(seq, n, k, Q);
    int64_t cnt = orc_query_keys(o, Q, (uint64_t)nw, out, cap);
    free(Q);
    return cnt;
}

/* Batch of queries.  kind 0: keys[offsets[q]..offsets[q+1]) are query q's
 * terms; kind 1: bases[offsets[q]..offsets[q+1]) is query q's sequence.
 * Inputs are validated first; the lowest-numbered bad query decides the
 * returned error and is stored in *bad_query.  On success counts[q] holds
 * |A_q| and, if ids != NULL and the total fits in ids_cap, ids holds the
 * concatenated ascending lists; *total gets the total either way.  Queries
 * are spread over nthreads OpenMP threads (each query is computed alone). */
int orc_query_batch(const orc_t *o, int kind, const void *data, const uint64_t *offsets,
                    uint64_t nq, uint32_t k, int nthreads, uint64_t *counts,
                    uint32_t *ids, uint64_t ids_cap, uint64_t *total, uint64_t *bad_query) {
    for (uint64_t q = 0; q < nq; ++q) {
        int rc = ORC_OK;
        if (offsets[q + 1] < offsets[q]) rc = ORC_EINVAL;
        else if (kind == 0) { if (offsets[q + 1] == offsets[q]) rc = ORC_EINVAL; }
        else {
            int64_t nw = orc_kmers((const uint8_t *)data + offsets[q], offsets[q + 1] - offsets[q], k, NULL);
            if (nw < 0) rc = (int)nw;
            else if (nw == 0) rc = ORC_EBADSEQ;
        }
        if (rc) { if (bad_query) *bad_query = q; return rc; }
    }
    uint32_t **res = (uint32_t **)calloc(nq ? nq : 1, sizeof(uint32_t *));
    if (!res) return ORC_ENOMEM;
    if (nthreads < 1) nthreads = 1;
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        orc_scratch sc;
        int ok = scratch_init(o, &sc) == ORC_OK;
        uint64_t qcap = 1 << 16;
        uint64_t *Q = (uint64_t *)malloc(sizeof(uint64_t) * qcap);
        uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * (o->K ? o->K : 1));
        if (!Q || !buf) ok = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t qi = 0; qi < (int64_t)nq; ++qi) {
            if (!ok) { failed = 1; continue; }
            uint64_t q = (uint64_t)qi;
            const uint64_t *terms;
            uint64_t nt;
            if (kind == 0) {
                terms = (const uint64_t *)data + offsets[q];
                nt = offsets[q + 1] - offsets[q];
            } else {
                uint64_t n = offsets[q + 1] - offsets[q];
                uint64_t most = n - (k & 0xffu) + 1;  /* every window; fewer with ORC_SKIPN */
                if (most > qcap) {
                    free(Q);
                    qcap = most;
                    Q = (uint64_t *)malloc(sizeof(uint64_t) * qcap);
                    if (!Q) { ok = 0; failed = 1; continue; }
                }
                nt = (uint64_t)orc_kmers((const uint8_t *)data + offsets[q], n, k, Q);
                terms = Q;
            }
            int64_t c = query_terms(o, terms, nt, &sc, buf, o->K);
            counts[q] = (uint64_t)c;
            res[q] = (uint32_t *)malloc(sizeof(uint32_t) * (c ? (uint64_t)c : 1));
            if (!res[q]) { failed = 1; continue; }
            memcpy(res[q], buf, sizeof(uint32_t) * (uint64_t)c);
        }
        free(Q); free(buf);
        scratch_free(&sc);
    }
    uint64_t tot = 0;
    for (uint64_t q = 0; q < nq && !failed; ++q) tot += counts[q];
    if (total) *total = tot;
    if (!failed && ids && tot <= ids_cap) {
        uint64_t at = 0;
        for (uint64_t q = 0; q < nq; ++q) {
            memcpy(ids + at, res[q], sizeof(uint32_t) * counts[q]);
            at += counts[q];
        }
    }
    for (uint64_t q = 0; q < nq; ++q) free(res[q]);
    free(res);
    return failed ? ORC_ENOMEM : ORC_OK;
}

/* ---------------- folding over (appendix) ---------------- */

/* OR cell b + B/2 onto cell b of every table and halve B: each new cell is the
 * Bloom filter of the union of the two old cells' sets. */
int orc_fold(orc_t *o) {
    if (o->B < 2 || (o->B & 1)) return ORC_EINVAL;
    const uint32_t B2 = o->B / 2;
    uint64_t *nb = (uint64_t *)calloc((size_t)o->R * B2 * o->wpb, sizeof(uint64_t));
    if (!nb) return ORC_ENOMEM;
    for (uint32_t r = 0; r < o->R; ++r)
        for (uint32_t b = 0; b < B2; ++b) {
            const uint64_t *lo = bf_of(o, r, b), *hi = bf_of(o, r, b + B2);
            uint64_t *dst = nb + ((uint64_t)r * B2 + b) * o->wpb;
            for (uint64_t w = 0; w < o->wpb; ++w) dst[w] = lo[w] | hi[w];
        }
    free(o->bits);
    o->bits = nb;
    o->B = B2;
    return build_members(o);
}

/* OR another structure with identical parameters into this one (the merge of
 * node-local structures built from disjoint sets, Sec. 5.2). */
int orc_merge(orc_t *o, const orc_t *src) {
    if (o->K != src->K || o->B != src->B || o->R != src->R || o->m != src->m || o->eta != src->eta ||
        o->seed != src->seed || o->B_local != src->B_local || o->n_nodes != src->n_nodes ||
        o->a_tau != src->a_tau || o->c_tau != src->c_tau)
        return ORC_EINVAL;
    for (uint64_t w = 0; w < (uint64_t)o->R * o->B * o->wpb; ++w) o->bits[w] |= src->bits[w];
    for (uint64_t w = 0; w < (o->K + 63) / 64; ++w) o->reg[w] |= src->reg[w];
    return ORC_OK;
}

/* ---------------- inspection ---------------- */

/* Copies the m bits of BF(table r, cell b) as ceil(m/64) little-endian words
 * (bit p of the filter = bit p&63 of word p>>6). */
void orc_export_bf(const orc_t *o, uint32_t r, uint32_t b, uint64_t *out) {
    memcpy(out, bf_of(o, r, b), sizeof(uint64_t) * o->wpb);
}

/* Bit `pos` of every cell of table r: bit b of the result (word b>>6) is bit
 * pos of BF(r, b).  out must hold ceil(B/64) words. */
void orc_get_row(const orc_t *o, uint32_t r, uint64_t pos, uint64_t *out) {
    memset(out, 0, sizeof(uint64_t) * ((o->B + 63) / 64));
    for (uint32_t b = 0; b < o->B; ++b) {
        const uint64_t *bf = bf_of(o, r, b);
        if ((bf[pos >> 6] >> (pos & 63)) & 1ULL) out[b >> 6] |= 1ULL << (b & 63);
    }
}

/* Number of set bits of each BF, out[r*B + b]. */
void orc_cell_popcount(const orc_t *o, uint64_t *out) {
    for (uint32_t r = 0; r < o->R; ++r)
        for (uint32_t b = 0; b < o->B; ++b) {
            const uint64_t *bf = bf_of(o, r, b);
            uint64_t c = 0;
            for (uint64_t w = 0; w < o->wpb; ++w) c += (uint64_t)__builtin_popcountll(bf[w]);
            out[(uint64_t)r * o->B + b] = c;
        }
}

void orc_export_reg(const orc_t *o, uint64_t *out) {
    memcpy(out, o->reg, sizeof(uint64_t) * ((o->K + 63) / 64));
}
