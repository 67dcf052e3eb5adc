// k_build_bucket.cu -- construction (Algorithm 1, Sec. 3.1) with every key
// hashed once per input chunk.
//
// The windowed build (k_build.cu) keeps one L2-sized slice of the rows
// resident while the whole input streams past, so every key is extracted and
// hashed once per window.  Here a scatter pass hashes each key of a chunk of
// the input once, turns every (table, hash) bit it sets into a 4-byte update
// record -- the bit's offset inside its window of the rows -- and files the
// records into one bucket per window (a block-local counting sort in shared
// memory, then one reservation per window and block).  An apply pass then
// takes the windows one at a time and ORs their records into the rows with
// fire-and-forget atomics, so each window stays resident in L2 while it is
// written.  Setting bits is order-free, so the bits equal every other build's.
#include "rambo_impl.cuh"

namespace rgb {

constexpr int BK_THREADS = 256;
constexpr uint32_t BK_TILE_RECORDS = 8192;  // records staged per block per step
constexpr uint32_t BK_MAX_WINDOWS = 4096;

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

// Window of global row g.  With magic != 0 (all rows below 2^32, set by the
// launcher) the quotient is the high word of magic * g, magic = ceil(2^64 /
// rows_per_win): exact for every 32-bit g and divisor (Lemire, Kaser and
// Kurz, "Faster remainder by direct computation", 2019).
__device__ __forceinline__ uint32_t bk_window(uint64_t g, uint64_t rows_per_win, uint64_t magic) {
    return magic ? (uint32_t)__umul64hi(magic, g) : (uint32_t)(g / rows_per_win);
}

// Scatter: each step, thread i of the block takes kt consecutive key
// positions starting at p0 + i*kt and stages their records (with their
// windows) in shared memory.  The block counts the records per window, scans
// the counts into block-local offsets, reserves each window's share of its
// bucket with one atomic, and places every record at its window's offset in
// a second shared array, so the records leave for their buckets as runs of
// consecutive words (coalesced stores).  A bucket that would overflow sets
// *overflow instead (the caller then files the chunk again).
__global__ void __launch_bounds__(BK_THREADS) k_bucket_scatter(IndexView ix, HashParams hp, BatchView b,
                                                                uint64_t p_lo, uint64_t p_hi, uint32_t kt,
                                                                uint64_t rows_per_win, uint64_t magic, uint32_t n_win,
                                                                uint64_t cap, uint32_t* __restrict__ rec,
                                                                unsigned long long* __restrict__ fill,
                                                                unsigned long long* overflow, const DevStatus* st) {
    extern __shared__ __align__(16) unsigned char bk_smem[];
    uint32_t* s_rec = reinterpret_cast<uint32_t*>(bk_smem);                       // [BK_TILE_RECORDS] staged
    uint32_t* s_srt = s_rec + BK_TILE_RECORDS;                                     // [BK_TILE_RECORDS] by window
    unsigned long long* s_base = reinterpret_cast<unsigned long long*>(s_srt + BK_TILE_RECORDS);  // [n_win]
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_base + n_win);                // [n_win]
    uint32_t* s_off = s_cnt + n_win;                                               // [n_win]
    uint32_t* s_wsum = s_off + n_win;                                              // [BK_THREADS / 32]
    uint16_t* s_win = reinterpret_cast<uint16_t*>(s_wsum + BK_THREADS / 32);       // [BK_TILE_RECORDS] staged
    uint16_t* s_swin = s_win + BK_TILE_RECORDS;                                    // [BK_TILE_RECORDS] by window
    if (st->err != NO_ERR) return;
    const uint32_t R = ix.R, eta = ix.eta;
    const uint32_t per_key = R * eta;
    const uint32_t slots = kt * per_key;  // records a thread stages per step
    const uint64_t span = (uint64_t)kt * blockDim.x;
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // each thread scans a contiguous run of the window counters
    const uint32_t wper = (n_win + blockDim.x - 1) / blockDim.x;
    const uint32_t wlo = min(n_win, threadIdx.x * wper), whi = min(n_win, wlo + wper);
    for (uint64_t p0 = p_lo + blockIdx.x * span; p0 < p_hi; p0 += (uint64_t)gridDim.x * span) {
        for (uint32_t w = threadIdx.x; w < n_win; w += blockDim.x) s_cnt[w] = 0;
        // this thread's keys: positions q0 .. q0 + kt
        const uint64_t q0 = p0 + (uint64_t)threadIdx.x * kt;
        uint32_t* my_rec = s_rec + threadIdx.x * slots;
        uint16_t* my_win = s_win + threadIdx.x * slots;
        uint32_t nrec = 0;
        // the item holding the warp's first position (one search per warp);
        // each lane walks forward from it to its own
        const uint64_t wq0 = p0 + (uint64_t)(threadIdx.x & ~31u) * kt;
        uint64_t t = 0;
        if (lane == 0 && wq0 < p_hi) t = bk_find_item(b.offsets, b.n, wq0 + b.off0);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (q0 < p_hi) {
            uint64_t t_end = __ldg(b.offsets + t + 1) - b.off0;
            for (uint32_t u = 0; u < kt; ++u) {
                const uint64_t p = q0 + u;
                if (p >= p_hi) break;
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
                        const uint32_t win = bk_window(g, rows_per_win, magic);
                        const uint64_t row_in = g - (uint64_t)win * rows_per_win;
                        my_rec[nrec] = (uint32_t)(((row_in * ix.S + (cell >> 5)) << 5) | (cell & 31));
                        my_win[nrec] = (uint16_t)win;
                        ++nrec;
                    }
                }
            }
        }
        __syncthreads();
        for (uint32_t i = 0; i < nrec; ++i) atomicAdd(&s_cnt[my_win[i]], 1u);
        __syncthreads();
        // block-local exclusive offsets of the windows, and each window's
        // share of its bucket reserved with one atomic
        uint32_t run = 0;
        for (uint32_t w = wlo; w < whi; ++w) run += s_cnt[w];
        uint32_t incl = run;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= (unsigned)off) incl += y;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        uint32_t before = incl - run;
        for (unsigned v = 0; v < wid; ++v) before += s_wsum[v];
        for (uint32_t w = wlo; w < whi; ++w) {
            const uint32_t c = s_cnt[w];
            s_off[w] = before;
            before += c;
            s_base[w] = c ? atomicAdd(fill + w, (unsigned long long)c) : 0ull;
            s_cnt[w] = 0;  // reused as the running slot of each window
        }
        __syncthreads();
        uint32_t total = 0;
        for (unsigned v = 0; v < BK_THREADS / 32; ++v) total += s_wsum[v];
        for (uint32_t i = 0; i < nrec; ++i) {
            const uint32_t w = my_win[i];
            const uint32_t at = s_off[w] + atomicAdd(&s_cnt[w], 1u);
            s_srt[at] = my_rec[i];
            s_swin[at] = (uint16_t)w;
        }
        __syncthreads();
        // runs of one window's records go out as consecutive words
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
            const uint32_t w = s_swin[i];
            const unsigned long long at = s_base[w] + (i - s_off[w]);
            if (at < cap) rec[(uint64_t)w * cap + at] = s_srt[i];
            else *overflow = 1;
        }
        __syncthreads();  // staging and counters are rewritten by the next step
    }
}

// Apply window `win`: OR its bucket's records into the rows.
__global__ void __launch_bounds__(BK_THREADS) k_bucket_apply(uint32_t* __restrict__ rows, uint64_t win_word0,
                                                              const uint32_t* __restrict__ rec,
                                                              const unsigned long long* __restrict__ fill,
                                                              uint32_t win, uint64_t cap) {
    const uint64_t n = min((unsigned long long)cap, fill[win]);
    const uint32_t* r = rec + (uint64_t)win * cap;
    uint32_t* base = rows + win_word0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldcs(r + i);  // streamed once
        atomicOr(base + (x >> 5), 1u << (x & 31));
    }
}

size_t bucket_scatter_smem(uint32_t n_win) {
    // records staged and by window (4 + 4 bytes each), reserved bases, counts
    // and offsets per window, warp sums, and the records' windows (2 + 2 bytes)
    return (size_t)BK_TILE_RECORDS * 8 + (size_t)n_win * 16 + (BK_THREADS / 32) * 4 + (size_t)BK_TILE_RECORDS * 4;
}

uint32_t bucket_keys_per_thread(uint32_t R, uint32_t eta) {
    const uint32_t per_thread = BK_TILE_RECORDS / BK_THREADS;  // 32 record slots
    const uint32_t kt = per_thread / (R * eta);
    return kt < 1 ? 1 : kt;
}

cudaError_t launch_bucket_scatter(const IndexView& ix, const HashParams& hp, const BatchView& b, uint64_t p_lo,
                                  uint64_t p_hi, uint64_t rows_per_win, uint32_t n_win, uint64_t cap, uint32_t* rec,
                                  unsigned long long* fill, unsigned long long* overflow, const DevStatus* st,
                                  int num_sms, cudaStream_t s) {
    if (p_hi <= p_lo) return cudaSuccess;
    if (n_win > BK_MAX_WINDOWS || ix.R * ix.eta > BK_TILE_RECORDS / BK_THREADS) return cudaErrorInvalidValue;
    const uint32_t kt = bucket_keys_per_thread(ix.R, ix.eta);
    const size_t smem = bucket_scatter_smem(n_win);
    const void* f = reinterpret_cast<const void*>(&k_bucket_scatter);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t span = (uint64_t)kt * BK_THREADS;
    uint64_t blocks = (p_hi - p_lo + span - 1) / span;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, BK_THREADS, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t most = (uint64_t)num_sms * per_sm;
    if (blocks > most) blocks = most;
    // window quotients by multiplication when every global row is below 2^32
    const uint64_t rows_total = (uint64_t)ix.R * ix.m;
    const uint64_t magic =
        (rows_total <= (1ull << 32) && rows_per_win > 1) ? ~0ull / rows_per_win + 1 : 0ull;
    k_bucket_scatter<<<(unsigned)blocks, BK_THREADS, smem, s>>>(ix, hp, b, p_lo, p_hi, kt, rows_per_win, magic, n_win,
                                                                 cap, rec, fill, overflow, st);
    return cudaGetLastError();
}

cudaError_t launch_bucket_apply(uint32_t* rows, uint64_t win_word0, const uint32_t* rec,
                                const unsigned long long* fill, uint32_t win, uint64_t cap, int num_sms,
                                cudaStream_t s) {
    k_bucket_apply<<<(unsigned)(num_sms * 8), BK_THREADS, 0, s>>>(rows, win_word0, rec, fill, win, cap);
    return cudaGetLastError();
}

}  // namespace rgb
