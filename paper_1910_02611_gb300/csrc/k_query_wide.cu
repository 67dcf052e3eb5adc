// k_query_wide.cu -- the batched RAMBO query (Algorithm 2, Sec. 3.2, with the
// sequence rule of Sec. 3.2.1) for indexes whose rows are too wide, or whose
// tables too many, for the register-tiled kernel: the paper's stacked
// whole-genome index (B = 50000, R = 5, folded to 25000 / 12500 / 6250;
// Sec. 5.2) and its ClueWeb09 index (B = 2e4, R = 4; Sec. 5.3) have rows of
// 2.5-6.25 KB.
//
// One thread block answers one query at a time, taking query indices from
// the same device work queue (atomic ticket) as the other kernel.  The
// query's per-table cell masks M_r (B bits each) live in shared memory.
// Terms are taken QW_TERMS at a time: the block computes their R*eta row
// positions, then every thread ANDs its share of the row words (all tables
// and terms of the step: the rows are read coalesced across the block, each
// one a contiguous W-word run) into the masks.  After each step the block
// checks whether some table's mask is empty (then no set can hold every
// term: the first FALSE is conclusive, Sec. 3.2.1) and stops.
//
// Set stage: every registered ID i is tested against bit phi_r(i) of M_r for
// every table (the union over hit cells per table and the intersection
// across tables of Algorithm 2); the survivors are counted, a range of the
// staging arena is reserved, and a second pass writes them in ascending
// order with a block-wide ordered compaction.
#include "rambo_impl.cuh"

namespace rgb {

constexpr int QW_TERMS = 4;  // terms per step

// shared memory: masks [R][S] words, then positions [QW_TERMS][R][EMAX]
// (uint64), then control words
size_t query_wide_smem_bytes(uint32_t R, uint32_t S) {
    return (size_t)R * S * 4 + (size_t)QW_TERMS * RMAX * EMAX * 8 + 64 * 4;
}

__global__ void __launch_bounds__(QW_THREADS) k_query_wide(IndexView ix, HashParams hp, BatchView b, QueryOut o,
                                                           DevStatus* st) {
    extern __shared__ __align__(16) unsigned char qw_smem[];
    const uint32_t R = ix.R, S = ix.S, W = ix.W, eta = ix.eta;
    uint32_t* sM = reinterpret_cast<uint32_t*>(qw_smem);                             // [R][S]
    uint64_t* sPos = reinterpret_cast<uint64_t*>(qw_smem + (size_t)R * S * 4);       // [QW_TERMS][RMAX][EMAX]
    uint32_t* ctl = reinterpret_cast<uint32_t*>(sPos + QW_TERMS * RMAX * EMAX);     // control
    unsigned long long* ctl_q = reinterpret_cast<unsigned long long*>(ctl);         // [0..1] ticket
    unsigned long long* ctl_start = reinterpret_cast<unsigned long long*>(ctl + 2); // [2..3] staging start
    uint32_t* ctl_nz = ctl + 4;                                                      // [4] tables still non-empty
    uint32_t* ctl_act = ctl + 5;                                                     // [5..8] term valid flags
    uint32_t* warp_cnt = ctl + 16;                                                   // [16..23] per-warp counts

    bv_resolve(b);
    if (query_batch_rejected(b, st)) return;
    const unsigned tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned nthreads = blockDim.x, nwarps = nthreads >> 5;
    const uint32_t rmask = R >= 32 ? ~0u : ((1u << R) - 1u);
    const uint64_t RW = (uint64_t)R * W;
    unsigned long long probed = 0, rows_read = 0;

    for (;;) {
        if (tid == 0) *ctl_q = atomicAdd(&st->ticket, 1ull);
        __syncthreads();
        const unsigned long long t = *ctl_q;
        if (t >= b.n) break;
        const unsigned long long q = b.perm ? (unsigned long long)__ldg(b.perm + t) : t;
        const uint64_t a = __ldg(b.offsets + q) - b.off0;
        const uint64_t e = __ldg(b.offsets + q + 1) - b.off0;
        const uint64_t nkeys = b.seq ? (e - a - b.k + 1) : (e - a);  // >= 1 (validated)

        for (uint64_t f = tid; f < RW; f += nthreads) sM[(f / W) * S + f % W] = ~0u;
        bool alive = true;
        // Steps visit terms in a strided order: step s takes terms s, s +
        // nsteps, s + 2 nsteps, ... so the first steps sample the whole query
        // (a substitution makes k consecutive windows absent).
        const uint64_t nsteps = (nkeys + QW_TERMS - 1) / QW_TERMS;
        for (uint64_t s = 0; s < nsteps && alive; ++s) {
            // positions of this step's terms
            if (tid < QW_TERMS) {
                const uint64_t idx = s + (uint64_t)tid * nsteps;
                bool act = idx < nkeys;
                uint64_t key = 0;
                if (act) {
                    if (b.seq) {
                        act = !b.skipn || window_resolved(b.nmask, a + idx, b.k);
                        key = kmer_at(b.packed, a + idx, b.k);
                        if (b.canon) key = canonical_kmer(key, b.k);
                    } else {
                        key = __ldg(b.keys + a + idx);
                    }
                }
                ctl_act[tid] = act ? 1u : 0u;
                const uint64_t y = mix64(key);
                for (uint32_t r = 0; r < R; ++r)
                    for (uint32_t j = 0; j < eta; ++j)
                        sPos[(tid * RMAX + r) * EMAX + j] = (hp.s[r][j] * y) >> ix.shift;
            }
            if (tid == 0) *ctl_nz = 0;
            __syncthreads();
            unsigned nact = 0;
#pragma unroll
            for (int u = 0; u < QW_TERMS; ++u) nact += ctl_act[u];
            // every thread ANDs its words of every table over the step's terms
            uint32_t nz = 0;
            for (uint64_t f = tid; f < RW; f += nthreads) {
                const uint32_t r = (uint32_t)(f / W), w = (uint32_t)(f % W);
                const uint32_t* base = ix.rows + (uint64_t)r * ix.m * S + w;
                uint32_t x = sM[r * S + w];
#pragma unroll
                for (int u = 0; u < QW_TERMS; ++u) {
                    if (!ctl_act[u]) continue;
                    const uint64_t* pu = sPos + (u * RMAX + r) * EMAX;
                    for (uint32_t j = 0; j < eta; ++j) x &= __ldg(base + pu[j] * S);
                }
                sM[r * S + w] = x;
                if (x) nz |= 1u << (r & 31);
            }
            // tables with a set bit anywhere (R <= 16 fits one word)
            nz = __reduce_or_sync(0xffffffffu, nz);
            if (lane == 0 && nz) atomicOr(ctl_nz, nz);
            __syncthreads();
            probed += nact;
            rows_read += (unsigned long long)nact * R * eta;
            if ((*ctl_nz & rmask) != rmask) alive = false;
            __syncthreads();  // ctl words are rewritten by the next step
        }

        uint32_t count = 0;
        unsigned long long start = 0;
        if (alive) {
            // pass 1: count the registered sets hit in every table
            for (uint64_t i0 = 0; i0 < ix.K; i0 += nthreads) {
                const uint64_t i = i0 + tid;
                bool ok = i < ix.K && ((__ldg(ix.reg + (i >> 5)) >> (i & 31)) & 1u);
                if (ok) {
                    const uint16_t* ph = ix.phi + i * ix.ps;
                    for (uint32_t r = 0; r < R && ok; ++r) {
                        const uint32_t c = __ldg(ph + r);
                        ok = (sM[r * S + (c >> 5)] >> (c & 31)) & 1u;
                    }
                }
                count += (uint32_t)__syncthreads_count(ok);
            }
            if (tid == 0 && count) *ctl_start = atomicAdd(&st->cursor, (unsigned long long)count);
            __syncthreads();
            start = count ? *ctl_start : 0ull;
            if (count && start + count <= o.stage_cap) {
                // pass 2: the same test, survivors written in ascending order
                uint32_t at = 0;
                for (uint64_t i0 = 0; i0 < ix.K; i0 += nthreads) {
                    const uint64_t i = i0 + tid;
                    bool ok = i < ix.K && ((__ldg(ix.reg + (i >> 5)) >> (i & 31)) & 1u);
                    if (ok) {
                        const uint16_t* ph = ix.phi + i * ix.ps;
                        for (uint32_t r = 0; r < R && ok; ++r) {
                            const uint32_t c = __ldg(ph + r);
                            ok = (sM[r * S + (c >> 5)] >> (c & 31)) & 1u;
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (lane == 0) warp_cnt[wid] = __popc(bal);
                    __syncthreads();
                    uint32_t before = 0, total = 0;
                    for (unsigned v = 0; v < nwarps; ++v) {
                        const uint32_t c = warp_cnt[v];
                        if (v < wid) before += c;
                        total += c;
                    }
                    if (ok) o.stage[start + at + before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
                    at += total;
                    __syncthreads();  // warp counts are rewritten by the next chunk
                }
            }
        }
        if (tid == 0) {
            o.qcount[q] = count;
            o.qstart[q] = start;
        }
        __syncthreads();  // masks and control words are reused by the next query
    }
    if (tid == 0 && probed) atomicAdd(&st->keys_probed, probed);
    if (tid == 0 && rows_read) atomicAdd(&st->rows_read, rows_read);
}

int query_wide_blocks_per_sm(uint32_t R, uint32_t S) {
    const size_t smem = query_wide_smem_bytes(R, S);
    const void* f = reinterpret_cast<const void*>(&k_query_wide);
    if (smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, QW_THREADS, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_query_wide(const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                              int blocks, DevStatus* st, cudaStream_t s) {
    if (b.n == 0 && !b.desc) return cudaSuccess;
    const size_t smem = query_wide_smem_bytes(ix.R, ix.S);
    const void* f = reinterpret_cast<const void*>(&k_query_wide);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_query_wide<<<(unsigned)(blocks > 0 ? blocks : 1), QW_THREADS, smem, s>>>(ix, hp, b, o, st);
    return cudaGetLastError();
}

cudaError_t load_query_wide_kernel() {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(&k_query_wide));
}

}  // namespace rgb
