// k_query_one.cu -- the plain one-query-per-launch GPU query: the comparison
// kernel the batched path is measured against.  One thread block answers one
// query straight from its ASCII bases or keys (Algorithm 2 with the sequence
// rule of Sec. 3.2.1): every thread builds k-mers byte by byte, reads all
// R*eta rows of its terms and ANDs them into shared per-table masks with
// shared-memory atomics; then the block scans every set ID in order and
// writes the survivors with a block-wide ordered compaction.  No early exit,
// no packing pass, no work queue: the straightforward design.
#include "rambo_impl.cuh"

namespace rgb {

constexpr int Q1_THREADS = 256;

__device__ __forceinline__ int q1_code(unsigned ch) {
    unsigned u = ch | 0x20u;
    bool ok = (u == 'a') | (u == 'c') | (u == 'g') | (u == 't');
    unsigned x = (u >> 1) & 3u;
    return ok ? (int)(x ^ (x >> 1)) : -1;
}

__global__ void __launch_bounds__(Q1_THREADS)
    k_query_one(IndexView ix, HashParams hp, int seq, const uint8_t* __restrict__ bases,
                const uint64_t* __restrict__ keys, uint64_t len, uint32_t k, int canon, int skipn,
                uint32_t* __restrict__ out_ids, uint32_t* __restrict__ out_count, int* __restrict__ bad) {
    extern __shared__ uint32_t sM[];  // [R][W] masks, then [32] warp counts, then the valid-window count
    uint32_t* warp_cnt = sM + ix.R * ix.W;
    uint32_t* n_valid = warp_cnt + 32;
    const int tid = threadIdx.x;
    for (uint32_t w = tid; w < ix.R * ix.W; w += blockDim.x) sM[w] = ~0u;
    if (tid == 0) *n_valid = 0;
    __syncthreads();
    const uint64_t nkeys = seq ? (len >= k ? len - k + 1 : 0) : len;
    for (uint64_t t = tid; t < nkeys; t += blockDim.x) {
        uint64_t key = 0;
        if (seq) {
            bool resolved = true;
            for (uint32_t c = 0; c < k; ++c) {
                int v = q1_code(bases[t + c]);
                if (v < 0) {
                    resolved = false;
                    if (!skipn) *bad = 1;
                    v = 0;
                }
                key = key * 4 + (uint64_t)v;
            }
            if (skipn && !resolved) continue;  // skip-N: not a term
            if (skipn) atomicAdd(n_valid, 1u);
            if (canon) {
                uint64_t rc = 0;  // reverse complement, from the bytes again
                for (uint32_t c = 0; c < k; ++c) {
                    int v = q1_code(bases[t + k - 1 - c]);
                    rc = rc * 4 + (uint64_t)(3 - (v < 0 ? 0 : v));
                }
                if (rc < key) key = rc;
            }
        } else {
            key = keys[t];
        }
        const uint64_t y = mix64(key);
        for (uint32_t r = 0; r < ix.R; ++r) {
            const uint32_t* base = ix.rows + (uint64_t)r * ix.m * ix.S;
            for (uint32_t w = 0; w < ix.W; ++w) {
                uint32_t acc = ~0u;
                for (uint32_t j = 0; j < ix.eta; ++j) acc &= base[((hp.s[r][j] * y) >> ix.shift) * ix.S + w];
                if (acc != ~0u) atomicAnd(&sM[r * ix.W + w], acc);
            }
        }
    }
    __syncthreads();
    if (seq && skipn && *n_valid == 0) {  // no term at all: a bad sequence
        if (tid == 0) {
            *bad = 1;
            *out_count = 0;
        }
        return;
    }
    // set stage: every registered ID whose cell is hit in every table, in order
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    uint32_t count = 0;
    for (uint64_t i0 = 0; i0 < ix.K; i0 += blockDim.x) {
        const uint64_t i = i0 + tid;
        bool ok = i < ix.K && ((ix.reg[i >> 5] >> (i & 31)) & 1u);
        if (ok)
            for (uint32_t r = 0; r < ix.R; ++r) {
                const uint32_t b = ix.phi[i * ix.ps + r];
                ok &= (sM[r * ix.W + (b >> 5)] >> (b & 31)) & 1u;
            }
        const unsigned bal = __ballot_sync(FULL, ok);
        if (lane == 0) warp_cnt[wid] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int v = 0; v < nw; ++v) {
            if (v < wid) before += warp_cnt[v];
            total += warp_cnt[v];
        }
        if (ok) out_ids[count + before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
        count += total;
        __syncthreads();
    }
    if (tid == 0) *out_count = count;
}

cudaError_t launch_query_one(const IndexView& ix, const HashParams& hp, int seq, const uint8_t* bases,
                             const uint64_t* keys, uint64_t len, uint32_t k, int canon, int skipn, uint32_t* out_ids,
                             uint32_t* out_count, int* bad, cudaStream_t s) {
    const size_t smem = (size_t)(ix.R * ix.W + 33) * 4;
    if (smem > 48 * 1024) {  // wide rows: masks of R * W words
        const cudaError_t e =
            cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_query_one), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_query_one<<<1, Q1_THREADS, smem, s>>>(ix, hp, seq, bases, keys, len, k, canon, skipn, out_ids, out_count,
                                            bad);
    return cudaGetLastError();
}

}  // namespace rgb
