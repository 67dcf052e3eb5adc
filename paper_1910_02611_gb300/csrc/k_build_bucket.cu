// k_build_bucket.cu -- construction (Algorithm 1, Sec. 3.1) with the bit
// updates applied in shared memory.
//
// The windowed build (k_build.cu) keeps one L2-sized slice of the rows
// resident while the whole input streams past and sets bits with global
// atomics; the atomics, not the hashing, bound it.  Here the index words are
// cut into slices of 32768 words (128 KB).  A pass over up to 4096 slices
// hashes every key of the batch, turns each (table, hash) bit that falls in
// the pass's slices into a 4-byte update record -- the bit's offset inside
// its slice -- and files the records into one bucket per slice (a
// block-local counting sort in shared memory, then one reservation per slice
// and block).  An apply launch then gives every slice a thread block that
// loads the slice into shared memory, ORs its bucket into it with
// shared-memory atomics and writes it back once.  Setting bits is
// order-free, so the bits equal every other build's.
#include "rambo_impl.cuh"

namespace rgb {

constexpr int BK_THREADS = 256;
constexpr uint32_t BK_TILE_RECORDS = 8192;  // records staged per block per step
constexpr uint32_t BK_MAX_SLICES = 4096;    // buckets of one pass
constexpr int SLICE_LOG2 = 15;              // 32768 words = 128 KB per slice
constexpr uint32_t SLICE_WORDS = 1u << SLICE_LOG2;
constexpr int AP_THREADS = 1024;

uint32_t bucket_slice_words() { return SLICE_WORDS; }

// largest t in [0, n) with off[t] <= pos
__device__ __forceinline__ uint64_t bk_find_item(const uint64_t* __restrict__ off, uint64_t n, uint64_t pos) {
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (__ldg(off + mid) <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Scatter (rec != NULL) or count (rec == NULL): each step, thread i of the
// block takes kt consecutive key positions starting at p0 + i*kt and stages
// the records of its keys that fall in slices [s_lo, s_lo + n_sl); the block
// counts them per slice, reserves each slice's share of its bucket with one
// atomic on fill[], and writes them at bucket_off[slice] + slot.  A record
// past its bucket's end sets *overflow instead (the caller then counts the
// pass exactly and files it again).
__global__ void __launch_bounds__(BK_THREADS) k_bucket_scatter(IndexView ix, HashParams hp, BatchView b,
                                                                uint32_t kt, uint64_t s_lo, uint32_t n_sl,
                                                                const uint64_t* __restrict__ bucket_off,
                                                                uint32_t* __restrict__ rec,
                                                                unsigned long long* __restrict__ fill,
                                                                unsigned long long* overflow, const DevStatus* st) {
    extern __shared__ __align__(16) unsigned char bk_smem[];
    uint32_t* s_rec = reinterpret_cast<uint32_t*>(bk_smem);                       // [BK_TILE_RECORDS]
    uint16_t* s_sl = reinterpret_cast<uint16_t*>(s_rec + BK_TILE_RECORDS);        // [BK_TILE_RECORDS]
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_sl + BK_TILE_RECORDS);        // [n_sl]
    unsigned long long* s_base = reinterpret_cast<unsigned long long*>(s_cnt + ((n_sl + 1) & ~1u));  // [n_sl]
    if (st->err != NO_ERR) return;
    const uint32_t R = ix.R, eta = ix.eta;
    const uint32_t slots = kt * R * eta;  // records a thread stages per step (at most 32)
    const uint64_t span = (uint64_t)kt * blockDim.x;
    for (uint64_t p0 = blockIdx.x * span; p0 < b.total; p0 += (uint64_t)gridDim.x * span) {
        for (uint32_t w = threadIdx.x; w < n_sl; w += blockDim.x) s_cnt[w] = 0;
        const uint64_t q0 = p0 + (uint64_t)threadIdx.x * kt;
        uint32_t* my_rec = s_rec + threadIdx.x * slots;
        uint16_t* my_sl = s_sl + threadIdx.x * slots;
        uint32_t nrec = 0;
        // the item holding the warp's first position (one search per warp);
        // each lane walks forward from it to its own
        const uint64_t wq0 = p0 + (uint64_t)(threadIdx.x & ~31u) * kt;
        uint64_t t = 0;
        if ((threadIdx.x & 31) == 0 && wq0 < b.total) t = bk_find_item(b.offsets, b.n, wq0 + b.off0);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (q0 < b.total) {
            uint64_t t_end = __ldg(b.offsets + t + 1) - b.off0;
            for (uint32_t u = 0; u < kt; ++u) {
                const uint64_t p = q0 + u;
                if (p >= b.total) break;
                while (p >= t_end) {  // next item holding p (skips empty items)
                    ++t;
                    t_end = __ldg(b.offsets + t + 1) - b.off0;
                }
                if (b.seq && p + b.k > t_end) continue;  // window runs past the end of this set's sequence
                if (b.skipn && !window_resolved(b.nmask, p, b.k)) continue;
                uint64_t key;
                if (b.seq) {
                    key = kmer_at(b.packed, p, b.k);
                    if (b.canon) key = canonical_kmer(key, b.k);
                } else {
                    key = __ldg(b.keys + p);
                }
                const uint64_t y = mix64(key);
                const uint16_t* ph = ix.phi + __ldg(b.set_ids + t) * ix.ps;
                for (uint32_t r = 0; r < R; ++r) {
                    const uint32_t cell = ph[r];
                    for (uint32_t j = 0; j < eta; ++j) {
                        const uint64_t g = (uint64_t)r * ix.m + ((hp.s[r][j] * y) >> ix.shift);  // global row
                        const uint64_t gw = g * ix.S + (cell >> 5);                             // global word
                        const uint64_t sl = (gw >> SLICE_LOG2) - s_lo;
                        if (sl >= n_sl) continue;  // another pass's slice
                        my_rec[nrec] = ((uint32_t)(gw & (SLICE_WORDS - 1)) << 5) | (cell & 31);
                        my_sl[nrec] = (uint16_t)sl;
                        ++nrec;
                    }
                }
            }
        }
        __syncthreads();
        for (uint32_t i = 0; i < nrec; ++i) atomicAdd(&s_cnt[my_sl[i]], 1u);
        __syncthreads();
        for (uint32_t w = threadIdx.x; w < n_sl; w += blockDim.x) {
            const uint32_t c = s_cnt[w];
            s_base[w] = c ? atomicAdd(fill + w, (unsigned long long)c) : 0ull;
            s_cnt[w] = 0;  // reused as the running slot of each slice
        }
        __syncthreads();
        if (rec) {
            for (uint32_t i = 0; i < nrec; ++i) {
                const uint32_t w = my_sl[i];
                const unsigned long long at = s_base[w] + atomicAdd(&s_cnt[w], 1u);
                const uint64_t lo = __ldg(bucket_off + w), hi = __ldg(bucket_off + w + 1);
                if (at < hi - lo) rec[lo + at] = my_rec[i];
                else *overflow = 1;
            }
        }
        __syncthreads();  // staging and counters are rewritten by the next step
    }
}

// Apply: block b owns slice s_lo + b: the slice's words go to shared memory,
// its bucket's records are ORed in with shared-memory atomics, and the slice
// goes back to the rows.  Slices whose bucket is empty are left untouched.
__global__ void __launch_bounds__(AP_THREADS) k_bucket_apply(uint32_t* __restrict__ rows, uint64_t total_words,
                                                              uint64_t s_lo, const uint64_t* __restrict__ bucket_off,
                                                              const uint32_t* __restrict__ rec,
                                                              const unsigned long long* __restrict__ fill) {
    extern __shared__ __align__(16) uint32_t ap_slice[];  // [SLICE_WORDS]
    const uint32_t bk = blockIdx.x;
    const uint64_t lo = bucket_off[bk];
    const uint64_t n = min((unsigned long long)(bucket_off[bk + 1] - lo), fill[bk]);
    if (n == 0) return;
    const uint64_t w0 = (s_lo + bk) << SLICE_LOG2;
    const uint32_t nw = (uint32_t)min((uint64_t)SLICE_WORDS, total_words - w0);
    const uint32_t nv = (nw & 3u) ? 0u : nw / 4;  // whole slices (and aligned tails) move as 16-byte vectors
    uint4* sv = reinterpret_cast<uint4*>(ap_slice);
    const uint4* gv = reinterpret_cast<const uint4*>(rows + w0);
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) sv[i] = gv[i];
    for (uint32_t i = nv * 4 + threadIdx.x; i < nw; i += blockDim.x) ap_slice[i] = rows[w0 + i];
    __syncthreads();
    const uint32_t* r = rec + lo;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t x = __ldcs(r + i);  // streamed once
        atomicOr(&ap_slice[x >> 5], 1u << (x & 31));
    }
    __syncthreads();
    uint4* gw = reinterpret_cast<uint4*>(rows + w0);
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) gw[i] = sv[i];
    for (uint32_t i = nv * 4 + threadIdx.x; i < nw; i += blockDim.x) rows[w0 + i] = ap_slice[i];
}

size_t bucket_scatter_smem(uint32_t n_sl) {
    return (size_t)BK_TILE_RECORDS * 6 + (size_t)((n_sl + 1) & ~1u) * 4 + (size_t)n_sl * 8;
}

uint32_t bucket_keys_per_thread(uint32_t R, uint32_t eta) {
    const uint32_t per_thread = BK_TILE_RECORDS / BK_THREADS;  // 32 record slots
    const uint32_t kt = per_thread / (R * eta);
    return kt < 1 ? 1 : kt;
}

cudaError_t launch_bucket_scatter(const IndexView& ix, const HashParams& hp, const BatchView& b, uint64_t s_lo,
                                  uint32_t n_sl, const uint64_t* bucket_off, uint32_t* rec, unsigned long long* fill,
                                  unsigned long long* overflow, const DevStatus* st, int num_sms, cudaStream_t s) {
    if (b.total == 0 || n_sl == 0) return cudaSuccess;
    if (n_sl > BK_MAX_SLICES || ix.R * ix.eta > BK_TILE_RECORDS / BK_THREADS) return cudaErrorInvalidValue;
    const uint32_t kt = bucket_keys_per_thread(ix.R, ix.eta);
    const size_t smem = bucket_scatter_smem(n_sl);
    const void* f = reinterpret_cast<const void*>(&k_bucket_scatter);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t span = (uint64_t)kt * BK_THREADS;
    uint64_t blocks = (b.total + span - 1) / span;
    const uint64_t most = (uint64_t)num_sms * 4;
    if (blocks > most) blocks = most;
    k_bucket_scatter<<<(unsigned)blocks, BK_THREADS, smem, s>>>(ix, hp, b, kt, s_lo, n_sl, bucket_off, rec, fill,
                                                                 overflow, st);
    return cudaGetLastError();
}

cudaError_t launch_bucket_apply(uint32_t* rows, uint64_t total_words, uint64_t s_lo, uint32_t n_sl,
                                const uint64_t* bucket_off, const uint32_t* rec, const unsigned long long* fill,
                                cudaStream_t s) {
    if (n_sl == 0) return cudaSuccess;
    const size_t smem = (size_t)SLICE_WORDS * 4;
    const void* f = reinterpret_cast<const void*>(&k_bucket_apply);
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bucket_apply<<<n_sl, AP_THREADS, smem, s>>>(rows, total_words, s_lo, bucket_off, rec, fill);
    return cudaGetLastError();
}

}  // namespace rgb
