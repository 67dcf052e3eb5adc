/*
 * rambo.h -- C ABI of librambo, a GB300 (sm_103a) implementation of RAMBO
 * (Repeated And Merged BloOm filters; Gupta et al., arXiv 1910.02611) for
 * multiple set membership testing (MSMT, Sec. 1): given K sets S_0..S_{K-1}
 * of 64-bit keys and a query, return the IDs of the sets that contain it.
 *
 * Structure (Sec. 3): R tables ("repetitions") of B cells; a 2-universal
 * partition hash phi_r sends each set ID to one cell per table; each cell is a
 * Bloom filter (Sec. 2) of m = 2^L bits over the union of its sets, probed at
 * eta positions h_{r,j}(x).  Stored bit-sliced in device memory: one row of B
 * bits per (table r, position p), so one row read tests all B cells of a table.
 *
 * Hash specification (the paper only asks for universal / 2-universal hashes):
 *   SplitMix64 (Steele, Lea, Flood 2014) with state = seed draws, in order,
 *   a_r = 1 + next() mod (P-1), c_r = next() mod P for r < R, then
 *   s_{r,j} = next() | 1 for r < R, j < eta, where P = 2^61 - 1, and
 *     phi_r(i)   = ((a_r * i + c_r) mod P) mod B
 *     h_{r,j}(x) = (s_{r,j} * mix64(x) mod 2^64) >> (64 - L)
 *   mix64 being SplitMix64's output finalizer.  DNA k-mers (1 <= k <= 32) are
 *   keys of 2 bits per base, A/a=0 C/c=1 G/g=2 T/t=3, first base most
 *   significant; every length-k window of a sequence is one key (with
 *   RAMBO_KMER_CANONICAL in k: the smaller of the window's key and its
 *   reverse complement's, the complement of code c being 3 - c).
 *
 * Conventions for every entry point:
 *   - Return RAMBO_OK (0) or a negative RAMBO_E* code; rambo_strerror names it.
 *     A failed call leaves the index as it was (inputs are validated on the
 *     device before anything is written), except RAMBO_ECUDA, after which the
 *     handle should be destroyed.
 *   - `on_device` = 1: every pointer argument (inputs and caller-provided
 *     outputs) is device memory; 0: host memory (pageable or pinned; DNA
 *     batches of 1 MiB or more in pinned memory are read in place by the
 *     packing kernel over NVLink-C2C instead of being copied first).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue their work on it and return once it has finished (they
 *     synchronise the stream), so inputs may be freed on return.
 *   - CSR batches: item t is data[offsets[t] .. offsets[t+1]) (uint64
 *     offsets, n+1 of them, non-decreasing; offsets[0] need not be 0).
 *   - Results are ascending, duplicate-free uint32 set IDs per query, in CSR
 *     form.  Result pointers returned by the query calls point into an arena
 *     owned by the handle: device memory when on_device = 1, pinned host
 *     memory otherwise; they stay valid until the next query call on the
 *     same handle or rambo_destroy.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef RAMBO_H
#define RAMBO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rambo rambo_t;

enum {
    RAMBO_OK = 0,
    RAMBO_EINVAL = -1,   /* bad parameter, decreasing offsets, empty key query */
    RAMBO_ERANGE = -2,   /* set ID >= K */
    RAMBO_EBADSEQ = -3,  /* base outside ACGTacgt (without RAMBO_KMER_SKIP_N), or a
                            query sequence with no k-mer window */
    RAMBO_ENOMEM = -4,   /* device or pinned host allocation failed */
    RAMBO_ENOSPC = -5,   /* caller-provided output too small (see *needed) */
    RAMBO_ECUDA = -6,    /* a CUDA runtime call failed */
    RAMBO_ETIMEOUT = -7, /* reserved for a bounded device-side wait that gives up;
                            no kernel of this library waits on a flag, so no
                            call returns it */
    RAMBO_EIO = -8,      /* file error in save/load */
    RAMBO_ESTATE = -9,   /* call not valid in the object's current state */
    RAMBO_E2BIG = -10    /* request larger than a fixed capacity: a plan's
                            buffers, a server slot, or the scratch of
                            rambo_query_seq_batch_noalloc */
};

/* OR-ed into a k-mer length argument: every window's key is the smaller of
 * the window and its reverse complement (both DNA strands give one key). */
#define RAMBO_KMER_CANONICAL 0x100u
/* OR-ed into a k-mer length argument: a byte outside ACGTacgt (an unresolved
 * base such as N) no longer rejects the sequence; every window holding one
 * is skipped, and the sequence's keys are its other windows (Sec. 3.2.1's
 * sliding window over the resolved stretches of a read; the paper's
 * whole-genome k-mers, Sec. 5.2, come from such reads).  Inserts register a
 * set whose sequence has no valid window, with no keys; a query sequence
 * with no valid window is RAMBO_EBADSEQ.  Combines with
 * RAMBO_KMER_CANONICAL. */
#define RAMBO_KMER_SKIP_N 0x200u

/* Limits of this implementation.  Indexes with R <= 8 and rows of at most
 * 4096 cells are queried by the register-tiled kernel (one warp, or a few,
 * per query); wider rows (the paper's stacked B = 50000 index, Sec. 5.2, or
 * ClueWeb09's B = 2e4, Sec. 5.3) and more tables by a kernel that gives each
 * query a thread block, its masks in shared memory, and reads every row
 * coalesced across the block. */
#define RAMBO_MAX_R 16       /* repetitions (tables) */
#define RAMBO_MAX_ETA 4      /* hashes per Bloom filter */
#define RAMBO_MAX_B 65535    /* cells per table */
#define RAMBO_MAX_L 32       /* m = 2^L bits per Bloom filter */

typedef struct rambo_info {
    uint64_t K;            /* set-ID capacity */
    uint32_t B, R, eta, L; /* cells, tables, hashes, log2(m) */
    uint64_t m;            /* bits per Bloom filter */
    uint64_t seed;
    uint32_t row_words;    /* W = ceil(B/32): 32-bit words holding one row's B bits */
    uint32_t row_stride;   /* S >= W: words between consecutive rows in memory */
    uint64_t index_bytes;  /* R * m * S * 4 */
    uint64_t n_registered; /* sets inserted so far (ID registered) */
    uint32_t nodes;        /* two-level hash: nodes (1 = plain partition) */
    uint32_t cells_per_node;
    uint64_t tau_seed;
} rambo_info_t;

/* Creates an empty index (Sec. 3: R tables x B cells of m-bit Bloom filters,
 * all zero) for set IDs 0..K-1.  Constraints: 1 <= K <= 2^32, 1 <= B <=
 * RAMBO_MAX_B, 1 <= R <= RAMBO_MAX_R, 1 <= eta <= RAMBO_MAX_ETA, m a power of
 * two with 2 <= m <= 2^32.  Allocates the index (R*m*S*4 bytes) and the
 * partition table on the current CUDA device.  Errors: RAMBO_EINVAL,
 * RAMBO_ENOMEM, RAMBO_ECUDA.  *out receives the handle (owned by the caller,
 * released with rambo_destroy). */
int rambo_create(uint64_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta,
                 uint64_t seed, rambo_t **out);

/* The two-level hash of the paper's node-parallel construction (Sec. 5.2,
 * appendix): n_nodes node-local structures of cells_per_node cells stacked
 * into one of B = cells_per_node * n_nodes cells.  A set i is routed to node
 * tau(i) = ((a_tau i + c_tau) mod P) mod n_nodes (a_tau, c_tau drawn from
 * SplitMix64 at tau_seed as a_r, c_r are from seed) and lives in cell
 * cells_per_node * tau(i) + phi_r(i) of table r, phi_r having range
 * cells_per_node.  Handles created with the same arguments on different GPUs
 * or at different times, each inserting only the sets routed to "its" node,
 * OR together (rambo_merge) into exactly the index built at once. */
int rambo_create_stacked(uint64_t K, uint32_t cells_per_node, uint32_t n_nodes, uint32_t R, uint64_t m,
                         uint32_t eta, uint64_t seed, uint64_t tau_seed, rambo_t **out);
/* tau(set_id) of a stacked handle (0 for a plain one). */
uint32_t rambo_node_of(const rambo_t *h, uint64_t set_id);
/* ORs src's rows and registered sets into dst (identical parameters and
 * device required; RAMBO_EINVAL otherwise). */
int rambo_merge(rambo_t *dst, const rambo_t *src, void *stream);

/* Releases all device and host memory of the handle (NULL is ignored).
 * Destroy the handle's plans and servers first: their captured graphs point
 * into its memory. */
void rambo_destroy(rambo_t *h);

int rambo_get_info(const rambo_t *h, rambo_info_t *out);

/* Algorithm 1 (Sec. 3.1), for n_sets sets in one call: set t has ID
 * set_ids[t] and keys keys[offsets[t] .. offsets[t+1]); every key is inserted
 * into the Bloom filter of cell phi_r(set_ids[t]) of every table r.  An ID may
 * appear several times and in several calls (insertion only sets bits, so the
 * resulting bits do not depend on order or split).  Every listed ID becomes
 * registered (reported by queries), even with no keys.
 * Errors: RAMBO_ERANGE (an ID >= K), RAMBO_EINVAL (decreasing offsets). */
int rambo_insert_batch(rambo_t *h, const uint64_t *set_ids, const uint64_t *keys,
                       const uint64_t *offsets, uint64_t n_sets, int on_device,
                       void *stream);

/* Algorithm 1 for one set: inserts keys[0 .. n) into set set_id (same as
 * rambo_insert_batch with one item). */
int rambo_insert(rambo_t *h, uint64_t set_id, const uint64_t *keys, uint64_t n, int on_device,
                 void *stream);

/* Algorithm 1 for sets given as DNA: set t's keys are the k-mers of
 * bases[offsets[t] .. offsets[t+1]) (Sec. 5.2: overlapping windows, k = 31).
 * A sequence shorter than k contributes no keys but its ID is registered.
 * Errors: RAMBO_ERANGE, RAMBO_EINVAL (offsets, k outside [1,32]),
 * RAMBO_EBADSEQ (a byte outside ACGTacgt). */
int rambo_insert_seq_batch(rambo_t *h, const uint64_t *set_ids, const uint8_t *bases,
                           const uint64_t *offsets, uint64_t n_sets, uint32_t k,
                           int on_device, void *stream);

/* Algorithm 2 (Sec. 3.2) for a batch of conjunctive queries: query q's terms
 * are keys[offsets[q] .. offsets[q+1]); the answer is the IDs i of registered
 * sets such that, in every table r, every term is in the Bloom filter of cell
 * phi_r(i) (per table, the union of the hit cells' sets; across tables, the
 * intersection; across terms, the conjunction of Sec. 3.2.1).  Results: set
 * IDs of query q are (*ids)[(*id_offsets)[q] .. (*id_offsets)[q+1]), ascending.
 * Errors: RAMBO_EINVAL (decreasing offsets or a query with no terms). */
int rambo_query_batch(rambo_t *h, const uint64_t *keys, const uint64_t *offsets,
                      uint64_t n_queries, int on_device, const uint32_t **ids,
                      const uint64_t **id_offsets, void *stream);

/* Large sequence query (Sec. 3.2.1): query q is the DNA sequence
 * bases[offsets[q] .. offsets[q+1]); its terms are all its k-mers and the
 * answer is the sets that hold every one of them.  Errors: RAMBO_EBADSEQ (a
 * byte outside ACGTacgt, or a sequence shorter than k), RAMBO_EINVAL. */
int rambo_query_seq_batch(rambo_t *h, const uint8_t *bases, const uint64_t *offsets,
                          uint64_t n_queries, uint32_t k, int on_device,
                          const uint32_t **ids, const uint64_t **id_offsets,
                          void *stream);

/* Same as rambo_query_batch / rambo_query_seq_batch but the results go to
 * caller-owned buffers: ids (capacity ids_cap entries) and id_offsets
 * (n_queries + 1 entries), device or host per on_device.  If the results do
 * not fit, returns RAMBO_ENOSPC and stores the needed number of IDs in
 * *needed (ids untouched; the call may be repeated with a larger buffer). */
int rambo_query_batch_into(rambo_t *h, const uint64_t *keys, const uint64_t *offsets,
                           uint64_t n_queries, int on_device, uint32_t *ids,
                           uint64_t ids_cap, uint64_t *id_offsets, uint64_t *needed,
                           void *stream);
int rambo_query_seq_batch_into(rambo_t *h, const uint8_t *bases, const uint64_t *offsets,
                               uint64_t n_queries, uint32_t k, int on_device,
                               uint32_t *ids, uint64_t ids_cap, uint64_t *id_offsets,
                               uint64_t *needed, void *stream);

/* Sequence query that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * they query -- code that runs where cudaMalloc/cudaFree are forbidden or
 * would stall (a real-time serving thread, a host callback, a process whose
 * memory budget is fixed up front) -- but can still launch kernels.  It
 * computes exactly what rambo_query_seq_batch_into computes; every pointer
 * (bases, offsets, ids, id_offsets) is device memory owned by the caller.
 * Its working memory (2-bit packed bases, per-query counts and staged
 * answers) is one array of 30 MiB (31,459,072 bytes) in device global memory
 * on every GPU the library is used on, held until the process exits.
 * Limits: at most 2^19 queries, 2^25 bases (offsets[n] - offsets[0]) and
 * 4,194,304 staging words per call, where a query's answer takes the smaller
 * of its ID count and ceil(K/32) words (dense answers are staged as a K-bit
 * bitmap); larger requests return RAMBO_E2BIG before any kernel runs
 * (answers beyond the staging limit are detected after the query kernel and
 * also return RAMBO_E2BIG).  rambo_create and rambo_load, which allocate
 * anyway, do the set-up with the handle's device current: they look up the
 * array's device address (cudaGetSymbolAddress, which under lazy module
 * loading is also when the array is reserved on that device) and load every
 * kernel this call can launch, so the call itself neither allocates nor
 * loads code.  All calls share the one array: each
 * call first clears the counters that must start at zero, so results never
 * depend on earlier calls, but calls that overlap on the GPU (several streams
 * or threads at once) race on it and must be serialised by the caller.
 * Returns RAMBO_ENOSPC with *needed set when ids_cap is too small, and the
 * errors of rambo_query_seq_batch otherwise.  RAMBO_KMER_SKIP_N is not
 * accepted here (RAMBO_EINVAL): its per-base mask would need working memory
 * beyond the fixed array. */
int rambo_query_seq_batch_noalloc(rambo_t *h, const uint8_t *bases, const uint64_t *offsets,
                                  uint64_t n_queries, uint32_t k, uint32_t *ids, uint64_t ids_cap,
                                  uint64_t *id_offsets, uint64_t *needed, void *stream);

/* The plain one-query-per-launch kernel, kept as the measurement baseline of
 * the batched path (no counterpart in the paper, which runs one query at a
 * time on one CPU thread, Sec. 5.2).  For every query q one thread block is
 * launched on `stream` that answers Algorithm 2 (with Sec. 3.2.1 for
 * sequences) for q alone, without early exit, packing pass or work queue,
 * and writes its ascending IDs to ids + q*K and their number to counts[q].
 * kind 0: data = device uint64 keys; kind 1: data = device ASCII bases.
 * host_offsets (n+1 entries) are in host memory so the launch loop needs no
 * device reads; ids must hold n*K entries, counts n.  Returns after the last
 * launch has finished.  Errors: RAMBO_EINVAL (empty query, k outside
 * [1,32]), RAMBO_EBADSEQ (a byte outside ACGTacgt). */
int rambo_query_one_per_launch(rambo_t *h, int kind, const void *data, const uint64_t *host_offsets,
                               uint64_t n_queries, uint32_t k, uint32_t *ids, uint32_t *counts,
                               void *stream);

/* ---- Graph-captured query plans (no counterpart in the paper) ----
 * A plan owns device and pinned host buffers for batches of up to
 * max_queries queries, max_items input items (bases for kind 1, keys for
 * kind 0) and max_ids result IDs, and a CUDA graph captured once at creation
 * (descriptor upload, validation, packing, the persistent query kernel, scan,
 * gather, status copy).  Every launch replays that graph; the batch size is
 * read on the device, so no kernel is re-launched from the host and nothing
 * is allocated.  Plans of one handle may run concurrently on different
 * streams; none may run while the handle inserts.  Inputs of a plan batch
 * start at offset 0: offsets[0] = 0 and offsets[n] = n_items. */
typedef struct rambo_plan rambo_plan_t;
int rambo_plan_create(rambo_t *h, int kind, uint64_t max_queries, uint64_t max_items, uint64_t max_ids,
                      uint32_t k, rambo_plan_t **out);
void rambo_plan_destroy(rambo_plan_t *p);
/* The plan's input buffers: pinned host (filled by the caller, copied by a
 * launch with from_host = 1) and device (filled by the caller, from_host = 0). */
int rambo_plan_buffers(rambo_plan_t *p, void **host_data, uint64_t **host_offsets, void **dev_data,
                       uint64_t **dev_offsets);
/* Enqueues one batch of n_queries queries (n_items items) on `stream` and
 * returns at once.  RAMBO_ESTATE if the previous launch was not waited for,
 * RAMBO_E2BIG beyond capacity. */
int rambo_plan_launch(rambo_plan_t *p, uint64_t n_queries, uint64_t n_items, int from_host, void *stream);
/* 0 when the launched batch has finished, 1 while it runs, < 0 on error. */
int rambo_plan_poll(rambo_plan_t *p);
/* Waits for the batch; returns its ID lists (device buffers, or pinned host
 * copies when to_host = 1, copied on `stream`) in CSR form.  RAMBO_ENOSPC
 * (with *n_ids = IDs needed) when the results exceed max_ids, and the
 * validation errors of the query calls. */
int rambo_plan_wait(rambo_plan_t *p, int to_host, const uint32_t **ids, const uint64_t **id_offsets,
                    uint64_t *n_ids, void *stream);
/* Kernels one replay launches (inside the graph). */
int rambo_plan_launches_per_replay(const rambo_plan_t *p);
/* Work and time of the plan's last batch, valid after a successful
 * rambo_plan_wait (fields as in rambo_query_stats_t, defined below; the
 * counters come from the batch's own status block).  query_kernel_ms and
 * device_ms come from CUDA events that nodes of the captured graph record
 * around the query kernel and around the whole replay; both are 0 if the
 * batch ran on the graph without those nodes (see rambo_plan_set_timing). */
struct rambo_query_stats;
int rambo_plan_last_stats(const rambo_plan_t *p, struct rambo_query_stats *out);
/* A plan holds two captured graphs of the same work: one with event-record
 * nodes around the query kernel and the replay (the default; its batches
 * report query_kernel_ms and device_ms) and one without them, whose replays
 * start and finish a few microseconds sooner (latency-bound small batches,
 * the server's plans).  on = 1 selects the first, 0 the second; answers are
 * identical.  RAMBO_ESTATE while a batch is in flight, RAMBO_ECUDA when the
 * timed graph could not be captured (the plan then runs the plain one). */
int rambo_plan_set_timing(rambo_plan_t *p, int on);

/* ---- Continuous-batching server (no counterpart in the paper; uses Sec.
 * 3.1's streaming updates) ----
 * A worker thread owns the GPU side: up to `slots` graph-captured plans per
 * query kind in flight on their own streams.  Whenever a slot frees up it
 * takes every queued query of its kind that fits its buffers (admission by
 * device memory), so requests that arrive while others run are batched and
 * overlap on the device.  Inserts are ordering barriers: queries submitted
 * before an insert see the index without it, queries after it see it.  While
 * a server exists, no other call may use its handle. */
typedef struct rambo_server rambo_server_t;
typedef struct rambo_server_config {
    uint32_t slots;              /* plans in flight per query kind (1..16) */
    uint64_t max_batch_queries;  /* queries per batch */
    uint64_t max_batch_bases;    /* DNA bases per batch (0 = no sequence queries) */
    uint64_t max_batch_keys;     /* keys per batch (0 = no key queries) */
    uint64_t max_batch_ids;      /* result IDs per batch */
    uint32_t k;                  /* k-mer length of sequence queries and inserts */
    uint32_t idle_wait_us;       /* worker sleep when idle (0 = 20 us) */
} rambo_server_config_t;
typedef struct rambo_server_stats {
    uint64_t queries, batches, inserts, keys;
    double seconds;              /* first launch to last completion */
    uint64_t p50_ns, p99_ns, max_ns;  /* submit-to-result latency of queries */
    /* worker thread time: staging and launching batches, waiting for and
     * copying out finished batches, running inserts, idle */
    uint64_t admit_ns, finish_ns, insert_ns, idle_ns;
    /* queries whose batch was deferred (requeued) because pinned host memory
     * for its answers was refused */
    uint64_t deferred;
} rambo_server_stats_t;
int rambo_server_create(rambo_t *h, const rambo_server_config_t *cfg, rambo_server_t **out);
/* Queues one query (kind 0: n_items uint64 keys; kind 1: n_items ASCII
 * bases); copies the input.  RAMBO_E2BIG if larger than a whole slot. */
int rambo_server_submit(rambo_server_t *s, int kind, const void *data, uint64_t n_items, uint64_t *ticket);
/* Queues an insert batch (as rambo_insert_batch / rambo_insert_seq_batch). */
int rambo_server_submit_insert(rambo_server_t *s, int kind, const uint64_t *set_ids, const void *data,
                               const uint64_t *offsets, uint64_t n_sets, uint64_t *ticket);
/* Result of a ticket: RAMBO_OK with the ascending IDs (up to cap; with
 * RAMBO_ENOSPC and *n_ids set, call again with a larger buffer), 1 if still
 * pending and wait = 0, or the request's error (RAMBO_E2BIG when its answer
 * alone exceeds max_batch_ids).  A delivered result or error is forgotten.  Finished batches' answers wait in host memory until collected
 * (large ones in pooled pinned buffers shared by the batch's requests, small
 * ones in ordinary memory), so uncollected results keep that memory. */
int rambo_server_result(rambo_server_t *s, uint64_t ticket, int wait, uint32_t *ids, uint64_t cap,
                        uint64_t *n_ids, uint64_t *latency_ns);
/* Waits until every submitted request has completed. */
int rambo_server_drain(rambo_server_t *s);
int rambo_server_stats(rambo_server_t *s, rambo_server_stats_t *out);
int rambo_server_reset_stats(rambo_server_t *s);
/* Load generator: submits request i (kind kinds[i], bytes
 * bytes[byte_offsets[i] .. byte_offsets[i+1])) at arrival_ns[i] after the
 * call starts, from the calling thread; tickets[i] receives its ticket. */
int rambo_server_replay(rambo_server_t *s, const uint8_t *kinds, const uint8_t *bytes,
                        const uint64_t *byte_offsets, const uint64_t *arrival_ns, uint64_t n,
                        uint64_t *tickets);
/* When pinned host memory for a finished batch's answers is refused, the
 * server does not fail the batch: its queries go back to the front of the
 * queue and run again after a 200 us pause in admission (collected results
 * return buffers to the pool meanwhile); a query deferred 64 times fails with
 * RAMBO_ENOMEM.  This call makes the next n such allocations (answers above
 * 256 KB) be refused as if cudaMallocHost had failed -- a host-side fault
 * injection for testing that path (0 ends it; nothing on the GPU fails). */
int rambo_server_inject_alloc_failures(rambo_server_t *s, uint32_t n);
/* Finishes all queued work, stops the worker and frees the server. */
void rambo_server_destroy(rambo_server_t *s);

/* Copies the bit-sliced index to host memory: n_words must equal
 * R * m * row_stride; word (r*m + p)*row_stride + w holds bits 32w..32w+31 of
 * row (r, p), bit b of the row being bit p of the Bloom filter of cell b of
 * table r (padding words are zero).  Errors: RAMBO_EINVAL (wrong n_words). */
int rambo_export_index(const rambo_t *h, uint32_t *host_words, uint64_t n_words);

/* Copies the registered-set bitmap (ceil(K/32) words, bit i = set i) and
 * the partition table (K*R values, phi_r(i) at [i*R + r]) to host memory. */
int rambo_export_registered(const rambo_t *h, uint32_t *host_words, uint64_t n_words);
int rambo_export_partition(const rambo_t *h, uint16_t *host_phi, uint64_t n);

/* Parameter chooser (Sec. 4 analysis, Sec. 5.1 parameter selection; no GPU
 * involved).  Given K sets of mean size n_mean keys, a key multiplicity V
 * (sets per key), a target per-BFU false-positive rate p and a target
 * failure probability delta (probability of any wrong ID for a query), fills
 * *B with the query-time optimum sqrt(K V / eta) of Lemma 4.4 (at least 2,
 * at most RAMBO_MAX_B), *R with the smallest R meeting Lemma 4.2's bound
 * K (1 - (1-p)(1-1/B)^V)^R <= delta (at most RAMBO_MAX_R; RAMBO_ERANGE if
 * that is not enough), *m with the power of two at or above the Bloom-filter
 * size n ln(1/p) / (ln 2)^2 for the expected n = n_mean K / B keys per cell,
 * and *eta with round(ln 2 * m / n) clamped to [1, RAMBO_MAX_ETA]. */
int rambo_suggest_params(uint64_t K, double n_mean, double V, double p, double delta, uint32_t *B,
                         uint32_t *R, uint64_t *m, uint32_t *eta);

/* The same chooser sized from a sampled prefix of the stream, as Sec. 5.1
 * does: the mean number of distinct keys per set is measured on the first
 * n_sample sets (host memory, CSR: kind 0 = uint64 keys, kind 1 = ASCII DNA
 * whose keys are its k-mers under the k-mer length and flags k) and taken as
 * n_mean; the other arguments and outputs are those of rambo_suggest_params.
 * *n_mean (if not NULL) receives the measured mean.  Errors: RAMBO_EINVAL
 * (no sample, decreasing offsets, bad k, a sample without keys),
 * RAMBO_EBADSEQ (a byte outside ACGTacgt without RAMBO_KMER_SKIP_N), and
 * RAMBO_ERANGE as rambo_suggest_params.  No GPU involved. */
int rambo_suggest_params_from_sample(uint64_t K, int kind, const void *data, const uint64_t *offsets,
                                     uint64_t n_sample, uint32_t k, double V, double p, double delta,
                                     uint32_t *B, uint32_t *R, uint64_t *m, uint32_t *eta, double *n_mean);

/* Folding over (appendix, Sec. 5.2): ORs cell b + B/2 onto cell b of every
 * table, halving B (and the index) while R, m, eta and the hashes stay.  The
 * result is exactly the index that rambo_create with B/2 and the same seed
 * would have built from the same inserts, because the partition hash mod B
 * then mod B/2 equals the hash mod B/2 (for a stacked handle every set's
 * cell becomes its cell mod B/2).  Resets the query configuration.
 * Errors: RAMBO_EINVAL when B is odd or 1, RAMBO_ENOMEM, RAMBO_ESTATE while
 * a plan or server created from the handle exists (folding replaces the
 * device buffers their captured graphs read; nothing is launched). */
int rambo_fold(rambo_t *h, void *stream);

/* Number of set bits of every Bloom filter, out[r*B + b] (host memory, R*B
 * entries); fill/m is the quantity Sec. 2's false-positive formula predicts. */
int rambo_cell_popcount(const rambo_t *h, uint64_t *host_out, void *stream);

/* Work and time of the last query call on this handle.  keys_probed counts
 * the keys whose rows were read: once a query's per-table mask is empty its
 * answer is empty and its remaining keys are skipped (Sec. 3.2.1, the first
 * FALSE is conclusive).  Times come from CUDA events recorded on the call's
 * stream around the query kernel and around all of the call's kernels. */
typedef struct rambo_query_stats {
    uint64_t n_queries;
    uint64_t keys_submitted;
    uint64_t keys_probed;
    uint64_t rows_read;        /* index rows read */
    uint64_t n_results;        /* set IDs returned */
    uint64_t kernel_launches;  /* kernels this library launched for the call */
    float query_kernel_ms;
    float device_ms;
    uint64_t stage_queries[4];  /* queries that reached the set stage, by stage used:
                                 * [0] staged dense (large ID space), [1] dense,
                                 * [2] sparse, [3] union */
    uint64_t staged_words;      /* 32-bit words the query kernel wrote to the
                                 * staging arena: ID lists and set bitmaps */
} rambo_query_stats_t;

int rambo_last_query_stats(const rambo_t *h, rambo_query_stats_t *out);

/* Tuning knobs of the query kernel; results never depend on them.
 *   lanes_per_key G, words_per_lane V (V divides the row stride, G*V >= stride),
 *   warps_per_block (1, 2, 4 or 8; 0 = automatic: the largest block that
 *   keeps at least 85% of the most warps resident per SM),
 *   blocks_per_sm (0 = as many as fit),
 *   set_stage: 0 = auto, 1 = dense scan of the partition table,
 *              2 = sparse enumeration of the hit cells' members,
 *              3 = union of the hit cells' member bitmaps (complemented for
 *                  tables with most cells hit), per table, intersected,
 *   visit_order and l2_fetch_bytes as described in the struct. */
typedef struct rambo_query_config {
    uint32_t lanes_per_key;
    uint32_t words_per_lane;
    uint32_t warps_per_block;
    uint32_t blocks_per_sm;
    uint32_t set_stage;
    uint32_t visit_order;     /* 0 = keys in input order; 1 = strided: the warp's
                               * first step spreads its terms evenly over the
                               * query, so a run of absent k-mers (a substitution
                               * touches k consecutive windows) is met at once;
                               * 2 = strided, and the first step reads table 0
                               * alone before the other tables */
    uint32_t l2_fetch_bytes;  /* 0 = leave the context's L2 fetch granularity;
                               * 32/64/128 = set it for the query kernel and
                               * restore it afterwards */
    uint32_t cluster;         /* 1 = hand queries to warps grouped by their
                               * minimizer (smallest term hash), so overlapping
                               * queries run together and share cached rows */
    uint32_t row_load;        /* cache operator of the row reads: 0 = ld.global.nc,
                               * 1 = .cg, 2 = .cs, 3 = .lu, 4 = .cv,
                               * 5 = .nc with L1::no_allocate, 6 = .nc with the
                               * L2 prefetch-size hint L2::64B, 7 = 5 and 6
                               * (the default) */
    uint32_t warps_per_query; /* 1 = one warp per query; 2, 4, 8 = that many warps
                               * of a block share each query (its terms and its
                               * set stage), capped at warps_per_block; 0 = from
                               * the batch size: as many as the persistent grid
                               * can give every query of the batch at once (a
                               * small batch spreads each query over a block).
                               * Needs a set stage with a shared-memory bitmap
                               * (K <= 131072); otherwise one warp per query. */
    uint32_t host_chunks;     /* answers returned in host memory (the arena
                               * query calls with on_device = 0, batches of
                               * 65536 queries or more): the batch runs as this
                               * many chunks whose answers are copied while the
                               * next ones compute; 0 = automatic (4), 1 = one
                               * piece, copied at the end; at most 8 */
    uint32_t answer_staging;  /* how a query's answer waits in the staging
                               * arena before it is laid out in query order:
                               * 0 = automatic (as its K-bit set bitmap when it
                               * holds more IDs than the bitmap has 32-bit
                               * words, else as its ID list); 1 = always as
                               * the ID list; f = 2..64: as the bitmap only
                               * when it holds more than f times that many IDs */
} rambo_query_config_t;

int rambo_get_query_config(const rambo_t *h, rambo_query_config_t *out);
/* Errors: RAMBO_EINVAL for a combination the kernels do not implement. */
int rambo_set_query_config(rambo_t *h, const rambo_query_config_t *cfg);

/* Construction tiling (results never depend on it): mode 0 = choose per
 * call from the input and index sizes, 1 = always run the build window by
 * window (each window of tile_bytes of the index stays resident in L2 while
 * the input streams past), 2 = one pass with every update going to device
 * memory, 3 = hash every key once per input chunk, file its updates by
 * 48 MiB window of the index and apply them window by window while the
 * window is resident in L2 (needs R * eta <= 32; falls back to mode 1 when
 * device memory for the updates is short).  Mode 0 takes 3 for large builds.
 * tile_bytes = 0 keeps the current window size of mode 1 (128 MiB
 * initially). */
int rambo_set_build_tiling(rambo_t *h, uint64_t tile_bytes, int mode);

/* Lists the query-kernel configurations valid for this handle (at most cap),
 * returns how many there are. */
int rambo_list_query_configs(const rambo_t *h, rambo_query_config_t *out, int cap);

/* Autotuner: times every query-kernel configuration the handle supports
 * (lanes per key, words per lane, warps per block, visiting order, and, when
 * warps_per_query is 0 and the set stage keeps a shared-memory bitmap, also
 * two warps per query) on the given sample batch (kind and pointers as in the query calls), `reps` runs
 * each, keeps the configuration with the smallest device time, stores it in
 * the handle and in *best.  Results never depend on the choice. */
int rambo_autotune(rambo_t *h, int kind, const void *data, const uint64_t *offsets, uint64_t n_queries,
                   uint32_t k, int on_device, int reps, rambo_query_config_t *best, void *stream);

/* Checkpoint (no counterpart in the paper, which keeps its index in memory):
 * writes the parameters, the registered-set bitmap and the rows to a file;
 * rambo_load recreates an identical handle on the current device.
 * Errors: RAMBO_EIO, RAMBO_EINVAL (not a file written by rambo_save). */
int rambo_save(const rambo_t *h, const char *path);
int rambo_load(const char *path, rambo_t **out);

/* Measurement helper (no counterpart in the paper): every thread of
 * blocks x threads reads reads_per_thread random rows of a device buffer of
 * n_rows rows spaced row_words 32-bit words apart (the first
 * min(row_words, 4) words of each), as the query's row probes do, with the
 * cache operator row_load (as in rambo_query_config_t).  *ms gets the kernel
 * time.  Gives the random-row throughput ceiling of the device. */
int rambo_random_row_probe(const uint32_t *dev_buf, uint64_t n_rows, uint32_t row_words,
                           uint64_t reads_per_thread, uint32_t blocks, uint32_t threads,
                           uint64_t seed, uint32_t row_load, float *ms, void *stream);

/* The current CUDA context's L2 fetch granularity hint
 * (cudaLimitMaxL2FetchGranularity): stores the present value in *prev (if not
 * NULL) and, when bytes > 0, sets it to bytes (32, 64 or 128).  A context-wide
 * performance hint; results never depend on it. */
int rambo_l2_fetch_granularity(uint32_t bytes, uint32_t *prev);

/* Index of the item (query or set) that caused the last RAMBO_EINVAL,
 * RAMBO_ERANGE or RAMBO_EBADSEQ returned on this handle. */
uint64_t rambo_last_error_item(const rambo_t *h);

const char *rambo_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* RAMBO_H */
