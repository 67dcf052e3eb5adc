// rambo_impl.cuh -- internal declarations shared by the librambo translation
// units: device-side hash helpers, parameter blocks, kernel launchers.
//
// Everything here follows the hash/layout specification stated in
// include/rambo.h; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rambo.h"

namespace rgb {

constexpr int RMAX = RAMBO_MAX_R;
constexpr int EMAX = RAMBO_MAX_ETA;
// the register-tiled query kernel: at most RF tables, rows of at most
// FAST_MAX_S words (32 lanes x 4 words)
constexpr int RF = 8;
constexpr uint32_t FAST_MAX_S = 128;
// partition table row: 8 uint16 per set ID (16 B) for R <= 8, else 16 (32 B)
__host__ __device__ inline uint32_t phi_stride_for(uint32_t R) { return R <= 8 ? 8u : 16u; }
// true when an index needs the block-per-query kernel
__host__ __device__ inline bool query_is_wide(uint32_t R, uint32_t S) { return R > (uint32_t)RF || S > FAST_MAX_S; }
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long NO_ERR = ~0ull;

// Device error word: (index << 8) | priority; the smallest value wins, so the
// lowest-numbered bad item is reported.  Priorities, lowest first, follow the
// order in which items are checked: set ID range, offsets, content.
constexpr unsigned PRIO_ERANGE = 1;
constexpr unsigned PRIO_EINVAL = 2;
constexpr unsigned PRIO_EBADSEQ = 3;

struct DevStatus {
    unsigned long long err;          // see above; NO_ERR when clean
    unsigned long long bad_pos;      // lowest position of a byte outside ACGTacgt
    unsigned long long ticket;       // next query index handed out to a warp
    unsigned long long cursor;       // staged result IDs handed out so far
    unsigned long long keys_probed;  // keys whose rows were read
    unsigned long long rows_read;    // row reads issued
    unsigned long long spare[2];
    unsigned long long stage_count[4];   // surviving queries per set stage (1 dense, 2 sparse, 3 union)
    unsigned long long gather_ticket;    // next queries handed out to a gather warp
};

// Position multipliers s_{r,j}, passed by value so every warp reads them from
// the kernel-parameter bank (uniform across the warp).
struct HashParams {
    uint64_t s[RMAX][EMAX];
};

// SplitMix64's output finalizer (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// phi_r(i) = ((a*i + c) mod (2^61-1)) mod B, for a < 2^61, c < 2^61, i < 2^32.
// The 128-bit value a*i + c is folded with 2^64 = 8 and 2^61 = 1 (mod 2^61-1).
__host__ __device__ __forceinline__ uint32_t partition_hash(uint64_t a, uint64_t c, uint64_t i,
                                                            uint32_t B) {
    const uint64_t P = (1ull << 61) - 1;
    uint64_t lo = a * i;
#ifdef __CUDA_ARCH__
    uint64_t hi = __umul64hi(a, i);
#else
    uint64_t hi = (uint64_t)(((unsigned __int128)a * i) >> 64);
#endif
    lo += c;
    hi += (lo < c) ? 1 : 0;
    uint64_t h8 = hi << 3;               // hi < 2^29 here, so no bits are lost
    h8 = (h8 & P) + (h8 >> 61);
    uint64_t t = (lo & P) + (lo >> 61) + h8;  // < 2^63
    t = (t & P) + (t >> 61);
    if (t >= P) t -= P;
    return (uint32_t)(t % B);
}

// Key of the k-mer whose first base is base number p of a 2-bit packed stream
// (32 bases per word, base 32w+t in bits 63-2t..62-2t of word w).  Reads word
// p/32 and, when the window crosses into it, word p/32 + 1.
__device__ __forceinline__ uint64_t kmer_at(const uint64_t* __restrict__ packed, uint64_t p,
                                            uint32_t k) {
    const uint64_t wi = p >> 5;
    const uint32_t o = (uint32_t)(p & 31) * 2;
    uint64_t win = __ldg(packed + wi) << o;
    if (o) win |= __ldg(packed + wi + 1) >> (64 - o);
    return win >> (64 - 2 * k);
}

// Loads of one, two or four 32-bit words of an index row with a selectable
// cache operator: 0 = ld.global.nc (read-only path), 1 = .cg (L2 only),
// 2 = .cs (streaming, evict first), 3 = .lu (last use), 4 = .cv (uncached),
// 5 = ld.global.nc.L1::no_allocate, 6 = ld.global.nc with the L2 prefetch
// size hint .L2::64B, 7 = both.  The row data and results never depend on
// the choice; it only changes how the memory system fetches isolated rows.
__device__ __forceinline__ uint32_t ld_row1(const uint32_t* p, int kind) {
    switch (kind) {
        case 1: return __ldcg(p);
        case 2: return __ldcs(p);
        case 3: return __ldlu(p);
        case 4: return __ldcv(p);
        case 5: {
            uint32_t v;
            asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
            return v;
        }
        case 6: {
            uint32_t v;
            asm volatile("ld.global.nc.L2::64B.u32 %0, [%1];" : "=r"(v) : "l"(p));
            return v;
        }
        case 7: {
            uint32_t v;
            asm volatile("ld.global.nc.L1::no_allocate.L2::64B.u32 %0, [%1];" : "=r"(v) : "l"(p));
            return v;
        }
        default: return __ldg(p);
    }
}
__device__ __forceinline__ uint2 ld_row2(const uint32_t* p, int kind) {
    const uint2* q = reinterpret_cast<const uint2*>(p);
    switch (kind) {
        case 1: return __ldcg(q);
        case 2: return __ldcs(q);
        case 3: return __ldlu(q);
        case 4: return __ldcv(q);
        case 5: {
            uint2 v;
            asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(q));
            return v;
        }
        case 6: {
            uint2 v;
            asm volatile("ld.global.nc.L2::64B.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(q));
            return v;
        }
        case 7: {
            uint2 v;
            asm volatile("ld.global.nc.L1::no_allocate.L2::64B.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(q));
            return v;
        }
        default: return __ldg(q);
    }
}
__device__ __forceinline__ uint4 ld_row4(const uint32_t* p, int kind) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    switch (kind) {
        case 1: return __ldcg(q);
        case 2: return __ldcs(q);
        case 3: return __ldlu(q);
        case 4: return __ldcv(q);
        case 5: {
            uint4 v;
            asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(q));
            return v;
        }
        case 6: {
            uint4 v;
            asm volatile("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(q));
            return v;
        }
        case 7: {
            uint4 v;
            asm volatile("ld.global.nc.L1::no_allocate.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(q));
            return v;
        }
        default: return __ldg(q);
    }
}

// Reverse complement of a k-mer key (complement of code c is 3 - c): NOT,
// reverse the 2-bit groups of the word, keep the top 2k bits.
__device__ __forceinline__ uint64_t revcomp_kmer(uint64_t fwd, uint32_t k) {
    uint64_t x = __brevll(~fwd);  // reverses bits, so each 2-bit group comes out bit-swapped
    x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    return x >> (64 - 2 * k);
}

__device__ __forceinline__ uint64_t canonical_kmer(uint64_t fwd, uint32_t k) {
    const uint64_t rc = revcomp_kmer(fwd, k);
    return rc < fwd ? rc : fwd;
}

// 1 when none of the k bases starting at base p is unresolved (skip-N
// windows): nmask holds one bit per base, bit t of word w for base 32w + t.
// Reads word p/32 and the next one (k <= 32, so o + k <= 63).
__device__ __forceinline__ bool window_resolved(const uint32_t* __restrict__ nmask, uint64_t p, uint32_t k) {
    const uint64_t wi = p >> 5;
    const uint32_t o = (uint32_t)(p & 31);
    const uint64_t two = (uint64_t)__ldg(nmask + wi) | ((uint64_t)__ldg(nmask + wi + 1) << 32);
    return ((two >> o) & ((1ull << k) - 1)) == 0;
}

// k and the canonical / skip-N flags from a k-mer length argument; false when invalid
__host__ __device__ inline bool split_k(uint32_t kflags, uint32_t* k, int* canon, int* skipn = nullptr) {
    *k = kflags & 0xffu;
    *canon = (kflags & RAMBO_KMER_CANONICAL) ? 1 : 0;
    if (skipn) *skipn = (kflags & RAMBO_KMER_SKIP_N) ? 1 : 0;
    return *k >= 1 && *k <= 32 && !(kflags & ~(0xffu | RAMBO_KMER_CANONICAL | RAMBO_KMER_SKIP_N));
}

__device__ __forceinline__ void record_error(DevStatus* st, uint64_t index, unsigned prio) {
    atomicMin(&st->err, (unsigned long long)((index << 8) | prio));
}

// ---------------------------------------------------------------------------
// parameter blocks
// ---------------------------------------------------------------------------

struct IndexView {
    uint32_t* rows;        // [R][m][S] words
    uint64_t m;            // rows per table
    uint32_t R, eta, shift;  // shift = 64 - L
    uint32_t S, W;         // row stride / words holding bits
    uint64_t K;
    uint32_t B;
    const uint16_t* phi;   // [K][ps]
    uint32_t ps;           // partition-table row stride (phi_stride_for(R))
    uint32_t* reg;         // ceil(K/32) words
    const uint64_t* mem_off;  // [R*B + 1] offsets of each cell's registered members (sparse stage)
    const uint32_t* mem_ids;  // registered members of each cell (unordered)
    const uint4* mem_phi;     // partition row of each mem_ids entry, same order
    const uint32_t* mem_bits; // [R][B][ceil(K/32)] member bitmap of every cell (union set stage)
};

struct BatchView {
    int seq;                       // 0: 64-bit keys, 1: packed DNA
    const uint64_t* keys;          // item data, index 0 = offsets[0]
    const uint64_t* packed;        // packed bases, base 0 = offsets[0]
    const uint64_t* offsets;       // n+1 absolute offsets
    uint64_t off0;                 // offsets[0]
    uint64_t total;                // offsets[n] - offsets[0]
    uint64_t n;                    // items
    uint32_t k;
    int canon;                     // keys are canonical k-mers (min of both strands)
    int skipn;                     // windows holding an unresolved base are skipped
    const uint32_t* nmask;         // skip-N: one bit per packed base, set = unresolved
    const uint64_t* set_ids;       // insert batches only
    const uint32_t* perm;          // queries only: processing order (NULL = 0..n-1)
    int no_resolve;                // 1: the query kernel leaves the unresolved-base lookup to a
                                   // separate launch over the whole batch (this view is a slice)
    const uint64_t* desc;          // device descriptor {n, total} (offsets[0] = 0) read at
                                   // kernel start instead of n/total/off0; lets one captured
                                   // CUDA graph serve batches of any size up to its capacity
};

// Takes n, total and off0 from the device descriptor when there is one.
__device__ __forceinline__ void bv_resolve(BatchView& b) {
    if (b.desc) {
        b.n = b.desc[0];
        b.total = b.desc[1];
        b.off0 = 0;
    }
}

// When packing met a byte outside ACGTacgt, the item holding the lowest one
// gets an EBADSEQ error (binary search for the largest t with offsets[t] <=
// position).  One thread; b must be resolved (bv_resolve).
__device__ __forceinline__ void resolve_bad_base(const BatchView& b, DevStatus* st) {
    const unsigned long long p = *(volatile unsigned long long*)&st->bad_pos;
    if (p == NO_ERR || b.n == 0) return;
    const uint64_t abs_p = p + b.off0;
    uint64_t lo = 0, hi = b.n;  // invariant: answer in [lo, hi)
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (b.offsets[mid] <= abs_p) lo = mid;
        else hi = mid;
    }
    record_error(st, lo, PRIO_EBADSEQ);
}

// First thing of every query kernel: the item holding an unresolved base
// (if packing met one) is recorded by one thread, and every block leaves
// once any validation error is known.  Returns true when the batch is bad.
__device__ __forceinline__ bool query_batch_rejected(const BatchView& b, DevStatus* st) {
    const bool bad_base = b.seq && *(volatile unsigned long long*)&st->bad_pos != NO_ERR;
    if (bad_base && !b.no_resolve && blockIdx.x == 0 && threadIdx.x == 0) resolve_bad_base(b, st);
    return bad_base || *(volatile unsigned long long*)&st->err != NO_ERR;
}

// A query's answer is staged either as its ascending ID list (count words)
// or, when that list would be longer than the query's K-bit set bitmap, as
// the bitmap itself (bits_words words; the gather expands it): dense answers
// then cross the staging arena in K/8 bytes instead of 4 bytes per ID.
constexpr uint64_t QSTART_BITMAP = 1ull << 63;  // flag in qstart: staged as a bitmap
__host__ __device__ inline uint32_t stage_bits_words(uint64_t K) { return (uint32_t)((K + 31) / 32); }

struct QueryOut {
    uint32_t* stage;       // staging arena (32-bit words)
    uint64_t stage_cap;    // its capacity in words
    uint64_t* qstart;      // per query: first staged word (| QSTART_BITMAP when staged as a bitmap)
    uint32_t* qcount;      // per query: number of IDs
    uint32_t bits_words;   // ceil(K/32) when bitmap staging is allowed, else 0
    uint32_t bits_min;     // an answer of more IDs than this is staged as the bitmap
};

// Staging form for an ID space of K sets: staging 0 = bitmap above ceil(K/32)
// IDs, 1 = ID lists only, f >= 2 = bitmap above f * ceil(K/32) IDs.  A query
// then stages at most bits_min words.
inline void set_staging(QueryOut& o, uint64_t K, uint32_t staging) {
    if (staging == 1) {
        o.bits_words = 0;
        o.bits_min = 0xffffffffu;
        return;
    }
    o.bits_words = stage_bits_words(K);
    const uint64_t m = (uint64_t)o.bits_words * (staging >= 2 ? staging : 1);
    o.bits_min = m > 0xffffffffull ? 0xffffffffu : (uint32_t)m;
}

struct QueryTuning {
    int V, G;              // words per lane, lanes per key
    int warps_per_block;
    int blocks;            // grid size
    int set_stage;         // 1 dense, 2 sparse, 0 auto
    int batch;             // queries taken per ticket
    int order;             // 0 input order, 1 strided, 2 strided + table-0 screening
    int load_kind;         // cache operator of the row loads (see ld_row1)
    int group;             // warps per query: 0 = from the batch size on the device, else at most this
    int blocks_group;      // grid of the grouped instance (0: not used)
    unsigned long long group_warps;  // its warps, the budget the group size is chosen against
    int wide;              // 1: the block-per-query kernel (R > RF or rows wider than FAST_MAX_S words)
    uint32_t staging;      // answer staging form (see set_staging)
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------

// k_util.cu
cudaError_t launch_status_reset(DevStatus* st, cudaStream_t s);
cudaError_t launch_phi_init(uint16_t* phi, uint64_t K, uint32_t R, uint32_t B, const uint64_t* a, const uint64_t* c,
                            uint32_t B_local, uint32_t n_nodes, uint64_t a_tau, uint64_t c_tau, cudaStream_t s);
cudaError_t launch_or_words(uint32_t* dst, const uint32_t* src, uint64_t n, cudaStream_t s);
cudaError_t launch_validate_batch(const BatchView& b, uint64_t min_len, uint64_t K, DevStatus* st,
                                  cudaStream_t s);
// nmask (skip-N): one bit per base, total/32 + 2 words; unresolved bases are
// marked there instead of being reported as errors
cudaError_t launch_pack(const uint8_t* bases, uint64_t total, uint64_t* packed, uint64_t n_words,
                        DevStatus* st, cudaStream_t s, const uint64_t* desc = nullptr, uint32_t* nmask = nullptr);
// skip-N queries: a query with no window free of unresolved bases is EBADSEQ
cudaError_t launch_check_windows(const BatchView& b, DevStatus* st, cudaStream_t s);
cudaError_t launch_resolve_bad_base(const BatchView& b, DevStatus* st, cudaStream_t s);
cudaError_t launch_register(const BatchView& b, uint32_t* reg, DevStatus* st, cudaStream_t s);
cudaError_t launch_scan_counts(const uint32_t* counts, uint64_t n, uint64_t* offsets,
                               uint64_t* tmp, uint64_t tmp_words, cudaStream_t s, const uint64_t* n_dev = nullptr,
                               int* n_launched = nullptr, const uint64_t* base_dev = nullptr,
                               unsigned long long* total_out = nullptr);
uint64_t scan_tmp_words(uint64_t n);
cudaError_t launch_gather(const QueryOut& o, const uint64_t* id_offsets, uint64_t n, uint32_t* ids,
                          DevStatus* st, cudaStream_t s, const uint64_t* n_dev = nullptr,
                          uint64_t ids_cap = ~0ull);
// queries: validation and (bases != NULL) packing in one launch; n_words is
// the packed capacity (a descriptor batch packs total/32 + 2 words of it)
cudaError_t launch_intake(const BatchView& b, uint64_t min_len, uint64_t K, const uint8_t* bases, uint64_t* packed,
                          uint64_t n_words, uint32_t* nmask, DevStatus* st, cudaStream_t s);
cudaError_t launch_cell_popcount(const IndexView& ix, unsigned long long* out, cudaStream_t s);
cudaError_t launch_members(const IndexView& ix, uint64_t* mem_off, uint32_t* mem_ids, uint4* mem_phi,
                           uint32_t* fill, cudaStream_t s);
cudaError_t launch_member_bits(const IndexView& ix, uint32_t* mem_bits, cudaStream_t s);
cudaError_t launch_fold(const uint32_t* old_rows, uint64_t n_rows, uint32_t W, uint32_t S, uint32_t B2, uint32_t W2,
                        uint32_t S2, uint32_t* new_rows, cudaStream_t s);

cudaError_t launch_cluster_order(const BatchView& b, uint64_t* keys, uint32_t* hist, uint64_t* bucket_off,
                                 uint64_t* scan_tmp, uint64_t scan_tmp_words, uint32_t* perm, const DevStatus* st,
                                 cudaStream_t s);
constexpr uint32_t CLUSTER_BUCKETS = 1u << 16;

// k_build.cu
cudaError_t launch_insert(const IndexView& ix, const HashParams& hp, const BatchView& b,
                          uint64_t row_lo, uint64_t row_hi, DevStatus* st, int num_sms, cudaStream_t s);

// k_build_bucket.cu: hash-once construction (records filed by window, applied window by window)
cudaError_t launch_bucket_scatter(const IndexView& ix, const HashParams& hp, const BatchView& b, uint64_t p_lo,
                                  uint64_t p_hi, uint64_t rows_per_win, uint32_t n_win, uint64_t cap, uint32_t* rec,
                                  unsigned long long* fill, unsigned long long* overflow, const DevStatus* st,
                                  int num_sms, cudaStream_t s);
cudaError_t launch_bucket_apply(uint32_t* rows, uint64_t win_word0, const uint32_t* rec,
                                const unsigned long long* fill, uint32_t win, uint64_t cap, int num_sms,
                                cudaStream_t s);

// k_query*.cu
bool query_config_supported(int V, int G, uint32_t S);
uint32_t query_smem_words_per_warp(uint32_t R, uint32_t S, uint64_t K, int use_bitmap);
size_t query_group_smem_bytes(uint32_t R, uint32_t S, uint64_t K, int wpb, int group);
int query_max_blocks_per_sm(int V, int G, uint32_t eta, bool grouped, int warps_per_block, size_t smem_per_block);
unsigned query_group_size(uint64_t n, int group, unsigned wpb, uint64_t group_warps, int use_bitmap);
cudaError_t launch_query(const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                         const QueryTuning& t, int use_bitmap, DevStatus* st, cudaStream_t s,
                         int* n_launched = nullptr);

// k_query_wide.cu: block-per-query kernel for wide rows or many tables
constexpr int QW_THREADS = 256;
size_t query_wide_smem_bytes(uint32_t R, uint32_t S);
int query_wide_blocks_per_sm(uint32_t R, uint32_t S);
cudaError_t launch_query_wide(const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                              int blocks, DevStatus* st, cudaStream_t s);
cudaError_t load_query_wide_kernel();

// k_query_one.cu: the plain one-query-per-launch kernel
cudaError_t launch_query_one(const IndexView& ix, const HashParams& hp, int seq, const uint8_t* bases,
                             const uint64_t* keys, uint64_t len, uint32_t k, int canon, int skipn, uint32_t* out_ids,
                             uint32_t* out_count, int* bad, cudaStream_t s);

// rambo_api.cu: what the fixed-scratch entry point needs from a handle
int handle_query_view(rambo_t* h, uint64_t n, IndexView* ix, HashParams* hp, QueryTuning* t, int* use_bitmap,
                      int* device);
// rambo_api.cu: plans hold device pointers of their handle inside a captured
// graph; the handle keeps a list of them, refuses calls that would move those
// buffers while any is alive, and orphans them (plan_orphan, rambo_plan.cu)
// when it is destroyed first, so they neither launch nor touch it again
void handle_attach_plan(rambo_t* h, rambo_plan_t* p);
void handle_detach_plan(rambo_t* h, rambo_plan_t* p);
void plan_orphan(rambo_plan_t* p);
// rambo_api.cu: device address of the fixed scratch, found when the handle was created
unsigned char* handle_noalloc_base(const rambo_t* h);

// rambo_noalloc.cu: with the handle's device current, finds the device
// address of the fixed scratch array and loads every kernel the no-alloc
// query can launch (eta selects the query-kernel instances), so that its
// calls need no module loading later
int noalloc_setup(uint32_t eta, unsigned char** base);

// kernel loading (lazy module loading otherwise loads a kernel at its first launch)
cudaError_t load_util_kernels();
cudaError_t load_query_kernels(uint32_t eta);

// k_roofline.cu
cudaError_t launch_random_rows(const uint32_t* buf, uint64_t n_rows, uint32_t row_words,
                               uint64_t reads_per_thread, uint64_t seed, uint32_t* sink,
                               int blocks, int threads, int load_kind, cudaStream_t s);

}  // namespace rgb
