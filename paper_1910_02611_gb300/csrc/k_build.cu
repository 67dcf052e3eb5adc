// k_build.cu -- Algorithm 1 (insertion, Sec. 3.1) on the bit-sliced index.
//
// For every key x of set i, every table r and every hash j, bit phi_r(i) of
// row (r, h_{r,j}(x)) is set with a fire-and-forget atomicOr (the Bloom-filter
// insert of Sec. 2 applied to cell phi_r(i) of table r).  Setting bits is
// order-free, so the result does not depend on thread scheduling.
//
// Large builds are tiled: one launch only performs the atomics whose row lies
// in [row_lo, row_hi), a window sized to stay resident in L2, and the input is
// streamed once per window.  Streaming the input is far cheaper than the DRAM
// read-modify-write of a sector per random atomic that an untiled build would
// cost.  (Hashing every key once and streaming the 8-byte hashes to each
// window instead measured no faster: the hash stream evicts the window from
// L2.)
#include "rambo_impl.cuh"

namespace rgb {

constexpr uint64_t KEYS_PER_THREAD = 8;
constexpr uint64_t STARTS_PER_THREAD = 32;

// largest t in [0, n) with off[t] <= pos
__device__ __forceinline__ uint64_t find_item(const uint64_t* __restrict__ off, uint64_t n, uint64_t pos) {
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (__ldg(off + mid) <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Each warp takes one contiguous run of positions with its lanes
// interleaved (lane l: p0 + l, p0 + l + 32, ...), so a step's packed words,
// keys and phi rows are adjacent across the warp, and the set holding a
// position is found by one binary search per warp, then followed forward.
__global__ void __launch_bounds__(256) k_insert(IndexView ix, HashParams hp, BatchView b, uint64_t row_lo,
                                                uint64_t row_hi, int r_lo, int r_hi, const DevStatus* st) {
    if (st->err != NO_ERR) return;
    const unsigned lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t per_warp = ((b.total + nwarps - 1) / nwarps + 31) & ~31ull;
    const uint64_t w_begin = warp * per_warp;
    const uint64_t w_end = min(w_begin + per_warp, b.total);
    if (w_begin >= w_end) return;
    uint64_t t = 0;
    if (lane == 0) t = find_item(b.offsets, b.n, w_begin + b.off0);
    t = __shfl_sync(FULL, t, 0);
    uint64_t t_end = __ldg(b.offsets + t + 1) - b.off0;
    const int R = (int)ix.R;
    uint32_t cell[RMAX];
    {
        const uint16_t* ph = ix.phi + __ldg(b.set_ids + t) * ix.ps;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) cell[r] = r < R ? ph[r] : 0u;
    }
    for (uint64_t p = w_begin + lane; p < w_end; p += 32) {
        if (p >= t_end) {
            // advance to the item holding p (skips empty items)
            do {
                ++t;
                t_end = __ldg(b.offsets + t + 1) - b.off0;
            } while (p >= t_end);
            const uint16_t* ph = ix.phi + __ldg(b.set_ids + t) * ix.ps;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) cell[r] = r < R ? ph[r] : 0u;
        }
        if (b.seq && p + b.k > t_end) continue;  // window runs past the end of this set's sequence
        if (b.skipn && !window_resolved(b.nmask, p, b.k)) continue;  // skip-N: holds an unresolved base
        uint64_t key;
        if (b.seq) {
            key = kmer_at(b.packed, p, b.k);
            if (b.canon) key = canonical_kmer(key, b.k);
        } else {
            key = __ldg(b.keys + p);
        }
        const uint64_t y = mix64(key);
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            if (r < r_lo || r > r_hi) continue;
            const uint32_t word = cell[r] >> 5;
            const uint32_t bit = 1u << (cell[r] & 31);
            const uint64_t rbase = (uint64_t)r * ix.m;
#pragma unroll
            for (int j = 0; j < EMAX; ++j) {
                if (j >= (int)ix.eta) break;
                const uint64_t pos = (hp.s[r][j] * y) >> ix.shift;
                const uint64_t grow = rbase + pos;
                if (grow - row_lo < row_hi - row_lo) atomicOr(ix.rows + grow * ix.S + word, bit);
            }
        }
    }
}

cudaError_t launch_insert(const IndexView& ix, const HashParams& hp, const BatchView& b, uint64_t row_lo,
                          uint64_t row_hi, DevStatus* st, int num_sms, cudaStream_t s) {
    if (b.total == 0 || b.n == 0 || row_hi <= row_lo) return cudaSuccess;
    const uint64_t span = 32 * (b.seq ? STARTS_PER_THREAD : KEYS_PER_THREAD);
    const uint64_t nchunks = (b.total + span - 1) / span;  // warps wanted at most
    uint64_t blocks = (nchunks + 7) / 8;
    uint64_t cap = (uint64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    int r_lo = (int)(row_lo / ix.m);
    int r_hi = (int)((row_hi - 1) / ix.m);
    if (r_hi >= (int)ix.R) r_hi = (int)ix.R - 1;
    k_insert<<<(unsigned)blocks, 256, 0, s>>>(ix, hp, b, row_lo, row_hi, r_lo, r_hi, st);
    return cudaGetLastError();
}

}  // namespace rgb
