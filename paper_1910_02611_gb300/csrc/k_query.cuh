// k_query.cuh -- the batched RAMBO query kernel (Algorithm 2, Sec. 3.2, with
// the sequence rule of Sec. 3.2.1), as a template over its register tiling.
//
// A group of P warps answers one query at a time, taking query indices from a
// device work queue (an atomic ticket), so queries of very uneven length
// balance themselves across a persistent grid.  P = 1 for large batches; a
// batch too small to occupy every warp gives each query up to a whole block
// (P <= 8), whose warps split the query's steps and its set stage and meet at
// a hardware barrier of their own.
//
// Per query (terms Q = its keys, or the k-mers of its sequence):
//   A1/A2  each lane group (G lanes) takes one term per step, builds the key
//          (from 2-bit packed DNA for sequences) and its R*eta positions;
//   A3     every lane reads V consecutive words of each of the term's R*eta
//          rows (one coalesced vector read per probe; all reads of a step are
//          issued before any is used) and ANDs the eta rows of each table: the
//          result is the term's B-bit cell mask per table (bit b set = the
//          term is in the Bloom filter of cell b);
//   A4     masks are AND-reduced across the warp's terms and into the running
//          per-table mask M_r; as soon as some M_r is empty no set can hold
//          every term (Sec. 3.2.1: the first FALSE is conclusive) and the
//          query stops reading rows;
//   A5     a surviving query keeps the registered sets i with bit phi_r(i) of
//          M_r set in every table: per table the union of the hit cells'
//          sets, across tables the intersection (Algorithm 2).  Per query the
//          cheapest of three exact stages fills a shared-memory bitmap of the
//          ID space: "dense" scans the partition table over all IDs; "sparse"
//          enumerates the registered members of the hit cells of the table
//          with the fewest hit cells and tests the other tables; "union" ORs
//          the hit cells' member bitmaps per table and ANDs the tables;
//   A6     the bitmap is compacted in ascending ID order, with coalesced
//          stores, into a staging arena (one atomic reservation per query),
//          or, when the answer holds more IDs than the bitmap has words,
//          the bitmap itself is staged; a scan + gather then lays the lists
//          out in query order (expanding staged bitmaps).
#pragma once

#include "rambo_impl.cuh"

namespace rgb {

constexpr int QK_THREADS_MAX = 256;
// per-warp staging words: dense survivors, the union stage's cell lists, or
// the compaction's run of IDs.  256 rather than 512 lets a fourth 4-warp
// block fit an SM when the ID space is 1e5 sets (16 warps instead of 12):
// 6% faster on the document workload, unchanged elsewhere.
constexpr int QK_ID_CAP = 256;
constexpr int QK_CTL = 16;      // per-warp control words (a query group uses its first warp's)

__host__ __device__ inline uint32_t qk_bitmap_words(uint64_t K) { return (uint32_t)((K + 31) / 32); }

template <int V>
__device__ __forceinline__ void qk_load(const uint32_t* __restrict__ p, uint32_t (&out)[V], int kind) {
    if constexpr (V == 1) {
        out[0] = ld_row1(p, kind);
    } else if constexpr (V == 2) {
        uint2 t = ld_row2(p, kind);
        out[0] = t.x;
        out[1] = t.y;
    } else {
        uint4 t = ld_row4(p, kind);
        out[0] = t.x;
        out[1] = t.y;
        out[2] = t.z;
        out[3] = t.w;
    }
}

template <int G>
__device__ __forceinline__ uint32_t qk_and_groups(uint32_t x) {
    if constexpr (G == 1) {
        return __reduce_and_sync(FULL, x);
    } else {
#pragma unroll
        for (int off = G; off < 32; off <<= 1) x &= __shfl_xor_sync(FULL, x, off);
        return x;
    }
}

__device__ __forceinline__ bool qk_set_passes(const IndexView& ix, const uint32_t* sM, uint64_t i,
                                              int skip_r) {
    if (!((__ldg(ix.reg + (i >> 5)) >> (i & 31)) & 1u)) return false;
    uint4 ph = __ldg(reinterpret_cast<const uint4*>(ix.phi) + i);
    uint32_t cell[8] = {ph.x & 0xffffu, ph.x >> 16, ph.y & 0xffffu, ph.y >> 16,
                        ph.z & 0xffffu, ph.z >> 16, ph.w & 0xffffu, ph.w >> 16};
    bool ok = true;
#pragma unroll
    for (int r = 0; r < RF; ++r) {
        if (r < (int)ix.R && r != skip_r) {
            uint32_t b = cell[r];
            ok &= (sM[r * ix.S + (b >> 5)] >> (b & 31)) & 1u;
        }
    }
    return ok;
}

// Synchronises the P warps of a query group (P = 1: the warp alone).  Groups
// of a block use distinct hardware barriers 1..4 (0 is __syncthreads').
__device__ __forceinline__ void qk_group_sync(unsigned P, unsigned gi) {
    if (P == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gi + 1), "r"(P * 32) : "memory");
    }
}

// Warps per query for a batch of n queries: 1 if the set stage has no
// shared-memory bitmap or group == 1; a forced group size (group = 2, 4, 8)
// capped at the block; else (group = 0) the largest power of two up to the
// block whose P * n warps the group launch's grid (group_warps) holds at once.
__host__ __device__ inline unsigned qk_group_size(uint64_t n, int group, unsigned wpb, uint64_t group_warps,
                                                  int use_bitmap) {
    unsigned P = 1;
    if (!use_bitmap || group == 1) return 1;
    const unsigned cap = group ? ((unsigned)group < wpb ? (unsigned)group : wpb) : wpb;
    while (P * 2 <= cap && (group || (uint64_t)P * 2 * n <= group_warps)) P *= 2;
    return P;
}

// One warp per query (batches that fill the grid).  Kept apart from the
// grouped form below: sharing one body with it cost this path 10-25% in
// register allocation on the document and uneven workloads.
template <int V, int G, int ETA>
__device__ __forceinline__ void qk_warp_queries(const IndexView& ix, const HashParams& hp, const BatchView& b,
                                                const QueryOut& o, int set_stage, int batch,
                                                uint32_t smem_per_warp, int use_bitmap, int order, int load_kind,
                                                DevStatus* st) {
    extern __shared__ uint32_t qk_smem[];
    constexpr int KPS = 32 / G;  // terms per warp step
    const unsigned lane = threadIdx.x & 31;
    const unsigned grp = lane / G;
    const unsigned slot = lane % G;
    const uint32_t w0 = slot * V;
    const bool has_words = w0 < ix.S;
    const int R = (int)ix.R;
    const int eta = (int)ix.eta;
    const uint32_t rmask = (1u << R) - 1u;
    uint32_t* sM = qk_smem + (threadIdx.x >> 5) * smem_per_warp + QK_CTL;  // [R][S] running masks
    uint32_t* sIds = sM + R * ix.S;                                // [QK_ID_CAP]
    uint32_t* sBits = sIds + QK_ID_CAP;                            // [ceil(K/32)] sparse-stage bitmap
    const uint32_t bw = qk_bitmap_words(ix.K);
    const uint32_t* __restrict__ rows = ix.rows;

    if (use_bitmap)
        for (uint32_t w = lane; w < bw; w += 32) sBits[w] = 0;
    __syncwarp();

    unsigned long long probed = 0, rows_read = 0;
    for (;;) {
        unsigned long long q0 = 0;
        if (lane == 0) q0 = atomicAdd(&st->ticket, (unsigned long long)batch);
        q0 = __shfl_sync(FULL, q0, 0);
        if (q0 >= b.n) break;
        const unsigned long long q1 = min(q0 + (unsigned long long)batch, (unsigned long long)b.n);
        for (unsigned long long t = q0; t < q1; ++t) {
            const unsigned long long q = b.perm ? (unsigned long long)__ldg(b.perm + t) : t;
            const uint64_t a = __ldg(b.offsets + q) - b.off0;
            const uint64_t e = __ldg(b.offsets + q + 1) - b.off0;
            const uint64_t nkeys = b.seq ? (e - a - b.k + 1) : (e - a);  // >= 1 (validated)

            uint32_t M[RF][V];
#pragma unroll
            for (int r = 0; r < RF; ++r)
#pragma unroll
                for (int v = 0; v < V; ++v) M[r][v] = has_words ? ~0u : 0u;

            bool alive = true;
            // step s visits terms s*KPS + g (input order) or g*nsteps + s
            // (strided: the first step samples the whole query evenly).
            // With screening, the first step reads table 0 only (phase 0) and
            // the other tables for the same terms only if the query is still
            // alive (phase 1); a query holding an absent term usually dies in
            // phase 0 at eta rows per term instead of R*eta.
            const uint64_t nsteps = (nkeys + KPS - 1) / KPS;
            const bool screen = order >= 2 && R > 1;
            const uint64_t nphases = nsteps + (screen ? 1 : 0);
            for (uint64_t ph = 0; ph < nphases; ++ph) {
                const uint64_t s = screen ? (ph == 0 ? 0 : ph - 1) : ph;
                const int rlo = (screen && ph == 1) ? 1 : 0;
                const int rhi = (screen && ph == 0) ? 1 : R;
                const uint64_t idx = order ? (uint64_t)grp * nsteps + s : s * KPS + grp;
                // skip-N: a window holding an unresolved base is not a term
                const bool act = idx < nkeys && (!b.skipn || window_resolved(b.nmask, a + idx, b.k));
                uint64_t key = 0;
                if (act) {
                    if (b.seq) {
                        key = kmer_at(b.packed, a + idx, b.k);
                        if (b.canon) key = canonical_kmer(key, b.k);
                    } else {
                        key = __ldg(b.keys + a + idx);
                    }
                }
                const uint64_t y = mix64(key);
                // A3: issue every row read of this step, then combine
                uint32_t val[RF][ETA][V];
                const bool ld = act && has_words;
#pragma unroll
                for (int r = 0; r < RF; ++r) {
                    if (r >= rlo && r < rhi && ld) {
                        const uint32_t* rb = rows + (uint64_t)r * ix.m * ix.S + w0;
#pragma unroll
                        for (int j = 0; j < ETA; ++j) {
                            if (j < eta) {
                                const uint64_t pos = (hp.s[r][j] * y) >> ix.shift;
                                qk_load<V>(rb + pos * ix.S, val[r][j], load_kind);
                            }
                        }
                    }
                }
                uint32_t nz = 0;
#pragma unroll
                for (int r = 0; r < RF; ++r) {
                    if (r < R) {
                        uint32_t any = 0;
                        const bool probed_r = r >= rlo && r < rhi;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            uint32_t x = ~0u;
                            if (ld && probed_r) {
#pragma unroll
                                for (int j = 0; j < ETA; ++j)
                                    if (j < eta) x &= val[r][j][v];
                            }
                            if (probed_r) {
                                x = qk_and_groups<G>(x);  // A4: across this step's terms
                                M[r][v] &= x;             // and into the query's masks
                            }
                            any |= M[r][v];
                        }
                        if (any) nz |= 1u << r;
                    }
                }
                nz = __reduce_or_sync(FULL, nz);
                {
                    const unsigned nact = __popc(__ballot_sync(FULL, act && slot == 0));
                    if (!(screen && ph == 1)) probed += nact;  // the screened terms were counted in phase 0
                    rows_read += (unsigned long long)nact * (unsigned)(rhi - rlo) * (unsigned)eta;
                }
                if (nz != rmask) {
                    alive = false;
                    break;
                }
            }

            uint32_t count = 0;
            unsigned long long start = 0;
            if (alive) {
                // stage the masks: row words [w0, w0+V) of table r
                if (grp == 0 && has_words) {
#pragma unroll
                    for (int r = 0; r < RF; ++r)
                        if (r < R)
#pragma unroll
                            for (int v = 0; v < V; ++v) sM[r * ix.S + w0 + v] = M[r][v];
                }
                __syncwarp();
                // per-table hit-cell counts; the table with the fewest hit cells
                // gives the sparse stage its candidates
                uint32_t pc[RF];
                int rstar = 0;
                uint32_t pmin = 0xffffffffu;
#pragma unroll
                for (int r = 0; r < RF; ++r) {
                    uint32_t c = 0;
                    if (r < R && grp == 0 && has_words)
#pragma unroll
                        for (int v = 0; v < V; ++v) c += __popc(M[r][v]);
                    pc[r] = (r < R) ? __reduce_add_sync(FULL, c) : 0u;
                    if (r < R && pc[r] < pmin) {
                        pmin = pc[r];
                        rstar = r;
                    }
                }
                // A5 strategy (all give the same set): 1 dense scan of every ID,
                // 2 sparse enumeration of rstar's hit cells, 3 union of the
                // precomputed member bitmaps of the hit cells (or of the missed
                // cells, complemented, when a table is mostly hit).  Auto picks
                // the fewest warp-wide operations (Lemma 4.4's candidate term).
                int stage = set_stage;
                if (!use_bitmap) stage = 1;
                uint32_t list_total = 0;
#pragma unroll
                for (int r = 0; r < RF; ++r)
                    if (r < R) list_total += pc[r] * 2 > ix.B ? ix.B - pc[r] : pc[r];
                const bool union_ok = ix.mem_bits && list_total <= 2u * QK_ID_CAP;
                if (stage == 3 && !union_ok) stage = 1;
                if (stage == 0) {
                    const uint64_t kw = (ix.K + 31) / 32;
                    const uint64_t dense = kw * (uint64_t)(R + 2);
                    const uint64_t sparse = ((uint64_t)pmin * (ix.K / ix.B + 1) / 32 + pmin) * (uint64_t)(R + 3) + kw / 16;
                    uint64_t uni = ~0ull;
                    if (union_ok) {
                        uni = kw / 32 + 1;
#pragma unroll
                        for (int r = 0; r < RF; ++r) {
                            if (r >= R) continue;
                            const uint32_t cr = pc[r] < ix.B - pc[r] ? pc[r] : ix.B - pc[r];
                            uni += (uint64_t)cr * (kw / 32 + 1);
                        }
                    }
                    stage = (dense <= sparse && dense <= uni) ? 1 : (sparse <= uni ? 2 : 3);
                }
                if (lane == 0) atomicAdd(&st->stage_count[use_bitmap ? stage : 0], 1ull);
                if (use_bitmap) {
                    if (stage == 1) {
                        // dense: one ballot per 32 IDs becomes one bitmap word; four
                        // chunks per iteration so their table loads are in flight together
                        constexpr int DU = 4;
                        for (uint64_t i0 = 0; i0 < ix.K; i0 += 32 * DU) {
                            uint32_t regw[DU];
                            uint4 ph[DU];
#pragma unroll
                            for (int u = 0; u < DU; ++u) {
                                const uint64_t i = i0 + 32 * u + lane;
                                regw[u] = i < ix.K ? __ldg(ix.reg + (i >> 5)) : 0u;
                                ph[u] = i < ix.K ? __ldg(reinterpret_cast<const uint4*>(ix.phi) + i) : make_uint4(0, 0, 0, 0);
                            }
#pragma unroll
                            for (int u = 0; u < DU; ++u) {
                                const uint64_t i = i0 + 32 * u + lane;
                                bool ok = i < ix.K && ((regw[u] >> (i & 31)) & 1u);
                                const uint32_t cell[8] = {ph[u].x & 0xffffu, ph[u].x >> 16, ph[u].y & 0xffffu,
                                                          ph[u].y >> 16,     ph[u].z & 0xffffu, ph[u].z >> 16,
                                                          ph[u].w & 0xffffu, ph[u].w >> 16};
#pragma unroll
                                for (int r = 0; r < RF; ++r)
                                    if (r < R) ok &= (sM[r * ix.S + (cell[r] >> 5)] >> (cell[r] & 31)) & 1u;
                                const unsigned bal = __ballot_sync(FULL, ok);
                                if (lane == 0 && i0 + 32 * u < ix.K) sBits[(i0 >> 5) + u] = bal;
                            }
                        }
                    } else if (stage == 2) {
                        // sparse: the registered members of table rstar's hit cells,
                        // tested on the other tables.  Hit cells are taken one mask
                        // word (up to 32 cells) at a time; lane j holds cell j's
                        // member range, and the members of all those cells form one
                        // run of candidates, 128 per iteration, whose IDs and
                        // partition rows are two independent coalesced loads.
                        const uint32_t* cellmask = sM + rstar * ix.S;
                        const uint64_t cbase = (uint64_t)rstar * ix.B;
                        // large cells (64+ members on average): one hit cell at a
                        // time, its members read as a contiguous run
                        const bool by_cell = ix.K >= 64ull * ix.B;
                        for (uint32_t w = 0; by_cell && w < ix.W; ++w) {
                            uint32_t hits = cellmask[w];
                            while (hits) {
                                const uint64_t cell = cbase + w * 32 + (uint32_t)(__ffs(hits) - 1);
                                hits &= hits - 1;
                                const uint32_t m0 = (uint32_t)__ldg(ix.mem_off + cell);
                                const uint32_t m1 = (uint32_t)__ldg(ix.mem_off + cell + 1);
                                constexpr int SC = 4;
                                for (uint32_t u0 = m0; u0 < m1; u0 += 32 * SC) {
                                    uint32_t id[SC];
                                    uint4 ph[SC];
#pragma unroll
                                    for (int c = 0; c < SC; ++c) {
                                        const uint32_t pos = u0 + 32 * c + lane;
                                        const bool v = pos < m1;
                                        id[c] = v ? __ldg(ix.mem_ids + pos) : 0xffffffffu;
                                        ph[c] = v ? __ldg(ix.mem_phi + pos) : make_uint4(0, 0, 0, 0);
                                    }
#pragma unroll
                                    for (int c = 0; c < SC; ++c) {
                                        if (id[c] == 0xffffffffu) continue;
                                        const uint32_t cl[8] = {ph[c].x & 0xffffu, ph[c].x >> 16, ph[c].y & 0xffffu,
                                                                ph[c].y >> 16,     ph[c].z & 0xffffu, ph[c].z >> 16,
                                                                ph[c].w & 0xffffu, ph[c].w >> 16};
                                        bool ok = true;
#pragma unroll
                                        for (int r = 0; r < RF; ++r)
                                            if (r < R && r != rstar) ok &= (sM[r * ix.S + (cl[r] >> 5)] >> (cl[r] & 31)) & 1u;
                                        if (ok) atomicOr(sBits + (id[c] >> 5), 1u << (id[c] & 31));
                                    }
                                }
                            }
                        }
                        for (uint32_t w = 0; !by_cell && w < ix.W; ++w) {
                            const uint32_t hits = cellmask[w];
                            if (!hits) continue;
                            uint32_t m0 = 0, cnt = 0;
                            if ((hits >> lane) & 1u) {
                                const uint64_t cell = cbase + w * 32 + lane;
                                m0 = (uint32_t)__ldg(ix.mem_off + cell);
                                cnt = (uint32_t)__ldg(ix.mem_off + cell + 1) - m0;
                            }
                            uint32_t incl = cnt;
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                const uint32_t y = __shfl_up_sync(FULL, incl, off);
                                if (lane >= (unsigned)off) incl += y;
                            }
                            const uint32_t total = __shfl_sync(FULL, incl, 31);
                            const uint32_t base = m0 - (incl - cnt);  // list position of candidate u = base + u
                            constexpr int SU = 4;
                            for (uint32_t u0 = 0; u0 < total; u0 += 32 * SU) {
                                uint32_t id[SU];
                                uint4 ph[SU];
#pragma unroll
                                for (int c = 0; c < SU; ++c) {
                                    const uint32_t u = u0 + 32 * c + lane;
                                    // owner lane: the first lane whose inclusive count exceeds u
                                    uint32_t j = 0;
#pragma unroll
                                    for (uint32_t step = 16; step >= 1; step >>= 1) {
                                        const uint32_t e = __shfl_sync(FULL, incl, j + step - 1);
                                        if (e <= u) j += step;
                                    }
                                    const uint32_t pos = __shfl_sync(FULL, base, j) + u;
                                    const bool v = u < total;
                                    id[c] = v ? __ldg(ix.mem_ids + pos) : 0xffffffffu;
                                    ph[c] = v ? __ldg(ix.mem_phi + pos) : make_uint4(0, 0, 0, 0);
                                }
#pragma unroll
                                for (int c = 0; c < SU; ++c) {
                                    if (id[c] == 0xffffffffu) continue;
                                    const uint32_t cl[8] = {ph[c].x & 0xffffu, ph[c].x >> 16, ph[c].y & 0xffffu,
                                                            ph[c].y >> 16,     ph[c].z & 0xffffu, ph[c].z >> 16,
                                                            ph[c].w & 0xffffu, ph[c].w >> 16};
                                    bool ok = true;
#pragma unroll
                                    for (int r = 0; r < RF; ++r)
                                        if (r < R && r != rstar) ok &= (sM[r * ix.S + (cl[r] >> 5)] >> (cl[r] & 31)) & 1u;
                                    if (ok) atomicOr(sBits + (id[c] >> 5), 1u << (id[c] & 31));
                                }
                            }
                        }
                    } else {
                        // union of member bitmaps: G_r = OR of the hit cells' bitmaps
                        // (or NOT of the missed cells' when over half are hit); the
                        // answer is registered AND every G_r.  The cell lists go to
                        // shared memory first (warp prefix sums), then each lane ORs
                        // UW words per cell for UC cells at a time.
                        uint16_t* list = reinterpret_cast<uint16_t*>(sIds);
                        uint32_t list_off[RF + 1];
                        list_off[0] = 0;
#pragma unroll
                        for (int r = 0; r < RF; ++r) {
                            uint32_t n_r = 0;
                            if (r < R) {
                                const bool comp = pc[r] * 2 > ix.B;
                                for (uint32_t c0 = 0; c0 < ix.W; c0 += 32) {
                                    const uint32_t cw = c0 + lane;
                                    uint32_t bits = 0;
                                    if (cw < ix.W) {
                                        bits = comp ? ~sM[r * ix.S + cw] : sM[r * ix.S + cw];
                                        if (cw == ix.W - 1 && (ix.B & 31)) bits &= (1u << (ix.B & 31)) - 1u;
                                    }
                                    const uint32_t c = __popc(bits);
                                    uint32_t incl = c;
#pragma unroll
                                    for (int off = 1; off < 32; off <<= 1) {
                                        const uint32_t y = __shfl_up_sync(FULL, incl, off);
                                        if (lane >= (unsigned)off) incl += y;
                                    }
                                    uint32_t pos = list_off[r] + n_r + incl - c;
                                    while (bits) {
                                        list[pos++] = (uint16_t)(cw * 32 + (__ffs(bits) - 1));
                                        bits &= bits - 1;
                                    }
                                    n_r += __shfl_sync(FULL, incl, 31);
                                }
                            }
                            list_off[r + 1] = list_off[r] + n_r;
                        }
                        __syncwarp();
                        constexpr int UW = 4, UC = 4;
                        for (uint32_t wb = 0; wb < bw; wb += 32 * UW) {
                            uint32_t g[UW];
#pragma unroll
                            for (int u = 0; u < UW; ++u) {
                                const uint32_t w = wb + 32 * u + lane;
                                g[u] = w < bw ? __ldg(ix.reg + w) : 0u;
                            }
#pragma unroll
                            for (int r = 0; r < RF; ++r) {
                                if (r >= R) continue;
                                const bool comp = pc[r] * 2 > ix.B;
                                const uint32_t* mb = ix.mem_bits + (uint64_t)r * ix.B * bw;
                                uint32_t acc[UW] = {0, 0, 0, 0};
                                for (uint32_t t = list_off[r]; t < list_off[r + 1]; t += UC) {
                                    uint32_t v[UC][UW];
#pragma unroll
                                    for (int c = 0; c < UC; ++c) {
                                        const bool have = t + c < list_off[r + 1];
                                        const uint32_t* col = mb + (uint64_t)(have ? list[t + c] : 0) * bw;
#pragma unroll
                                        for (int u = 0; u < UW; ++u) {
                                            const uint32_t w = wb + 32 * u + lane;
                                            v[c][u] = (have && w < bw) ? __ldg(col + w) : 0u;
                                        }
                                    }
#pragma unroll
                                    for (int c = 0; c < UC; ++c)
#pragma unroll
                                        for (int u = 0; u < UW; ++u) acc[u] |= v[c][u];
                                }
#pragma unroll
                                for (int u = 0; u < UW; ++u) g[u] &= comp ? ~acc[u] : acc[u];
                            }
#pragma unroll
                            for (int u = 0; u < UW; ++u) {
                                const uint32_t w = wb + 32 * u + lane;
                                if (w < bw) sBits[w] = g[u];
                            }
                        }
                    }
                    __syncwarp();
                    // compaction: ascending IDs from the bitmap, bitmap cleared.
                    // 32 words (1024 IDs) at a time: lanes expand their word's bits
                    // into shared memory at their prefix position, then the warp
                    // copies the run out with coalesced stores.  An answer with
                    // more IDs than bitmap words is staged as the bitmap.
                    for (uint32_t w = lane; w < bw; w += 32) count += __popc(sBits[w]);
                    count = __reduce_add_sync(FULL, count);
                    // a dense answer is staged as the bitmap (fewer words)
                    const bool as_bits = count > o.bits_min && o.bits_words == bw;
                    const uint32_t words = as_bits ? bw : count;
                    if (lane == 0 && count) start = atomicAdd(&st->cursor, (unsigned long long)words);
                    start = __shfl_sync(FULL, start, 0);
                    const bool write = count && start + words <= o.stage_cap;
                    uint32_t at = 0;
                    if (as_bits) {
                        for (uint32_t w = lane; w < bw; w += 32) {
                            if (write) o.stage[start + w] = sBits[w];
                            sBits[w] = 0;
                        }
                        start |= QSTART_BITMAP;
                    }
                    for (uint32_t w0b = 0; w0b < bw && !as_bits; w0b += 32) {
                        const uint32_t w = w0b + lane;
                        uint32_t bits = (w < bw) ? sBits[w] : 0u;
                        uint32_t c = __popc(bits);
                        uint32_t incl = c;
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
                            uint32_t y = __shfl_up_sync(FULL, incl, off);
                            if (lane >= (unsigned)off) incl += y;
                        }
                        const uint32_t blk = __shfl_sync(FULL, incl, 31);
                        if (write && blk) {
                            uint32_t* dst = o.stage + start + at;
                            if (blk <= (uint32_t)QK_ID_CAP) {
                                uint32_t pos = incl - c;
                                while (bits) {
                                    sIds[pos++] = w * 32 + (__ffs(bits) - 1);
                                    bits &= bits - 1;
                                }
                                __syncwarp();
                                for (uint32_t t = lane; t < blk; t += 32) dst[t] = sIds[t];
                                __syncwarp();
                            } else {
                                uint32_t pos = incl - c;
                                while (bits) {
                                    dst[pos++] = w * 32 + (__ffs(bits) - 1);
                                    bits &= bits - 1;
                                }
                            }
                        }
                        if (w < bw) sBits[w] = 0;
                        at += blk;
                    }
                    __syncwarp();
                } else {
                    // ID space too large for a shared-memory bitmap: dense scan,
                    // survivors staged in shared memory, recounted if they overflow
                    for (uint64_t i0 = 0; i0 < ix.K; i0 += 32) {
                        const uint64_t i = i0 + lane;
                        const bool ok = (i < ix.K) && qk_set_passes(ix, sM, i, -1);
                        const unsigned bal = __ballot_sync(FULL, ok);
                        if (bal) {
                            const unsigned pre = __popc(bal & ((1u << lane) - 1u));
                            if (ok && count + pre < (uint32_t)QK_ID_CAP) sIds[count + pre] = (uint32_t)i;
                            count += __popc(bal);
                        }
                    }
                    if (lane == 0 && count) start = atomicAdd(&st->cursor, (unsigned long long)count);
                    start = __shfl_sync(FULL, start, 0);
                    if (count && start + count <= o.stage_cap) {
                        if (count <= (uint32_t)QK_ID_CAP) {
                            for (uint32_t t = lane; t < count; t += 32) o.stage[start + t] = sIds[t];
                        } else {
                            uint32_t at = 0;
                            for (uint64_t i0 = 0; i0 < ix.K; i0 += 32) {
                                const uint64_t i = i0 + lane;
                                const bool ok = (i < ix.K) && qk_set_passes(ix, sM, i, -1);
                                const unsigned bal = __ballot_sync(FULL, ok);
                                if (ok) o.stage[start + at + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
                                at += __popc(bal);
                            }
                        }
                    }
                }
            }
            if (lane == 0) {
                o.qcount[q] = count;
                o.qstart[q] = start;
            }
        }
    }
    if (lane == 0 && probed) atomicAdd(&st->keys_probed, probed);
    if (lane == 0 && rows_read) atomicAdd(&st->rows_read, rows_read);
}

// Two instances per tiling: GROUP = false is the one-warp-per-query kernel
// (P = 1 folded in at compile time), GROUP = true serves batches that give a
// query more than one warp.  A launch whose instance does not match the
// batch's group size returns at once, so a captured graph holds both and the
// batch size, read on the device, picks.  Tilings whose row words in flight
// (RF * ETA * V) fit in 64 registers are held to 128 registers a thread, so
// two full blocks share an SM; wider ones keep every register they need, and
// so does the one-warp V = 4, ETA = 2 tiling, measured 11% faster that way on
// the uneven workload (16-byte rows, 8 tables).
template <int V, int G, int ETA, bool GROUP>
__global__ void __launch_bounds__(QK_THREADS_MAX,
                                  (RF * ETA * V <= 64 && !(V == 4 && ETA == 2 && !GROUP)) ? 2 : 1)
    k_query(IndexView ix, HashParams hp, BatchView b, QueryOut o, int set_stage, int batch,
            uint32_t smem_per_warp, int use_bitmap, int order, int load_kind, int group,
            unsigned long long group_warps, DevStatus* st) {
    extern __shared__ uint32_t qk_smem[];
    constexpr int KPS = 32 / G;  // terms per warp step
    const unsigned lane = threadIdx.x & 31;
    const unsigned wid = threadIdx.x >> 5;
    const unsigned grp = lane / G;
    const unsigned slot = lane % G;
    const uint32_t w0 = slot * V;
    const bool has_words = w0 < ix.S;
    const int R = (int)ix.R;
    const int eta = (int)ix.eta;
    const uint32_t rmask = (1u << R) - 1u;
    const uint32_t bw = qk_bitmap_words(ix.K);
    const uint32_t* __restrict__ rows = ix.rows;

    bv_resolve(b);
    if (query_batch_rejected(b, st)) return;
    // Query group: P warps answer one query together (P = 1 for large
    // batches; up to 8 when the batch is too small to fill the grid, so a
    // lone query's steps and set stage spread over more warps).  group = 0
    // picks P from the batch size, else P = min(group, warps per block).
    const unsigned wpb = blockDim.x >> 5;
    const unsigned Pb = qk_group_size(b.n, group, wpb, group_warps, use_bitmap);
    if (GROUP != (Pb > 1)) return;  // the other instance serves this batch
    if constexpr (!GROUP) {
        qk_warp_queries<V, G, ETA>(ix, hp, b, o, set_stage, batch, smem_per_warp, use_bitmap, order, load_kind, st);
    } else {
        const unsigned P = Pb;
        const unsigned gi = wid / P, gw = wid % P;
        const bool leader = gw == 0 && lane == 0;
        // the group's shared state lives in its first warp's region; each warp
        // keeps its own staging words.  Layout of this instance: per warp
        // [QK_CTL] control, [R][S] masks, [QK_ID_CAP] staging (smem_per_warp
        // words, no bitmap), then one ceil(K/32)-word bitmap per query group
        // (groups have at least two warps, so half a bitmap per warp at most)
        uint32_t* lead = qk_smem + (gi * P) * smem_per_warp;
        uint32_t* ctl = lead;                                                // group control words
        uint32_t* sM = lead + QK_CTL;                                        // [R][S] running masks
        uint32_t* sBits = qk_smem + wpb * smem_per_warp + gi * ((bw + 3u) & ~3u);  // the group's bitmap
        uint32_t* sIds = qk_smem + wid * smem_per_warp + QK_CTL + R * ix.S;  // this warp's staging
        volatile unsigned long long* ctl_ticket = reinterpret_cast<volatile unsigned long long*>(ctl);
        volatile unsigned long long* ctl_start = reinterpret_cast<volatile unsigned long long*>(ctl + 2);
        volatile uint32_t* ctl_dead = ctl + 4;
        volatile uint32_t* ctl_cnt = ctl + 8;  // [8] per-warp counts

        // (groups only form when the set stage has a shared-memory bitmap)
        for (uint32_t w = gw * 32 + lane; w < bw; w += P * 32) sBits[w] = 0;
        batch = 1;
        qk_group_sync(P, gi);

        unsigned long long probed = 0, rows_read = 0;
        for (;;) {
            if (leader) *ctl_ticket = atomicAdd(&st->ticket, (unsigned long long)batch);
            qk_group_sync(P, gi);
            const unsigned long long q0 = *ctl_ticket;
            qk_group_sync(P, gi);
            if (q0 >= b.n) break;
            const unsigned long long q1 = min(q0 + (unsigned long long)batch, (unsigned long long)b.n);
            for (unsigned long long t = q0; t < q1; ++t) {
                const unsigned long long q = b.perm ? (unsigned long long)__ldg(b.perm + t) : t;
                const uint64_t a = __ldg(b.offsets + q) - b.off0;
                const uint64_t e = __ldg(b.offsets + q + 1) - b.off0;
                const uint64_t nkeys = b.seq ? (e - a - b.k + 1) : (e - a);  // >= 1 (validated)

                for (uint32_t w = gw * 32 + lane; w < (uint32_t)R * ix.S; w += P * 32) sM[w] = ~0u;
                if (leader) *ctl_dead = 0;
                qk_group_sync(P, gi);

                uint32_t M[RF][V];
#pragma unroll
                for (int r = 0; r < RF; ++r)
#pragma unroll
                    for (int v = 0; v < V; ++v) M[r][v] = has_words ? ~0u : 0u;

                bool alive = true;
                // Steps: step s visits terms s*KPS + g (input order) or g*nsteps + s
                // (strided: the first step samples the whole query evenly).  Warp
                // gw of the group takes steps gw, gw + P, ...  With screening, a
                // warp's first step reads table 0 only (phase 0) and the other
                // tables for the same terms only if the query is still alive
                // (phase 1); a query holding an absent term usually dies in phase
                // 0 at eta rows per term instead of R*eta.
                const uint64_t nsteps = (nkeys + KPS - 1) / KPS;
                const uint64_t mine = nsteps > gw ? (nsteps - gw + P - 1) / P : 0;  // steps of this warp
                const bool screen = order >= 2 && R > 1;
                const uint64_t nphases = mine + ((screen && mine) ? 1 : 0);
                for (uint64_t ph = 0; ph < nphases; ++ph) {
                    if (__shfl_sync(FULL, *ctl_dead, 0)) break;  // another warp found an empty table
                    const uint64_t s = gw + (uint64_t)P * (screen ? (ph == 0 ? 0 : ph - 1) : ph);
                    const int rlo = (screen && ph == 1) ? 1 : 0;
                    const int rhi = (screen && ph == 0) ? 1 : R;
                    const uint64_t idx = order ? (uint64_t)grp * nsteps + s : s * KPS + grp;
                    // skip-N: a window holding an unresolved base is not a term
                    const bool act = idx < nkeys && (!b.skipn || window_resolved(b.nmask, a + idx, b.k));
                    uint64_t key = 0;
                    if (act) {
                        if (b.seq) {
                            key = kmer_at(b.packed, a + idx, b.k);
                            if (b.canon) key = canonical_kmer(key, b.k);
                        } else {
                            key = __ldg(b.keys + a + idx);
                        }
                    }
                    const uint64_t y = mix64(key);
                    // A3: issue every row read of this step, then combine
                    uint32_t val[RF][ETA][V];
                    const bool ld = act && has_words;
#pragma unroll
                    for (int r = 0; r < RF; ++r) {
                        if (r >= rlo && r < rhi && ld) {
                            const uint32_t* rb = rows + (uint64_t)r * ix.m * ix.S + w0;
#pragma unroll
                            for (int j = 0; j < ETA; ++j) {
                                if (j < eta) {
                                    const uint64_t pos = (hp.s[r][j] * y) >> ix.shift;
                                    qk_load<V>(rb + pos * ix.S, val[r][j], load_kind);
                                }
                            }
                        }
                    }
                    uint32_t nz = 0;
#pragma unroll
                    for (int r = 0; r < RF; ++r) {
                        if (r < R) {
                            uint32_t any = 0;
                            const bool probed_r = r >= rlo && r < rhi;
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                uint32_t x = ~0u;
                                if (ld && probed_r) {
#pragma unroll
                                    for (int j = 0; j < ETA; ++j)
                                        if (j < eta) x &= val[r][j][v];
                                }
                                if (probed_r) {
                                    x = qk_and_groups<G>(x);  // A4: across this step's terms
                                    M[r][v] &= x;             // and into the query's masks
                                }
                                any |= M[r][v];
                            }
                            if (any) nz |= 1u << r;
                        }
                    }
                    nz = __reduce_or_sync(FULL, nz);
                    {
                        const unsigned nact = __popc(__ballot_sync(FULL, act && slot == 0));
                        if (!(screen && ph == 1)) probed += nact;  // the screened terms were counted in phase 0
                        rows_read += (unsigned long long)nact * (unsigned)(rhi - rlo) * (unsigned)eta;
                    }
                    if (nz != rmask) {
                        alive = false;
                        if (lane == 0) *ctl_dead = 1;
                        break;
                    }
                }

                // the query's masks in shared memory: row words [w0, w0+V) of table r
                // AND of the group's partial masks (a warp that stopped early
                // holds a superset, which the AND leaves correct)
                if (alive && mine && grp == 0 && has_words) {
#pragma unroll
                    for (int r = 0; r < RF; ++r)
                        if (r < R)
#pragma unroll
                            for (int v = 0; v < V; ++v) atomicAnd(sM + r * ix.S + w0 + v, M[r][v]);
                }
                qk_group_sync(P, gi);
                alive = *ctl_dead == 0;

                uint32_t count = 0;
                unsigned long long start = 0;
                // per-table hit-cell counts; the table with the fewest hit cells
                // gives the sparse stage its candidates
                uint32_t pc[RF];
                int rstar = 0;
                uint32_t pmin = 0xffffffffu;
                if (alive) {
#pragma unroll
                    for (int r = 0; r < RF; ++r) {
                        uint32_t c = 0;
                        if (r < R)
                            for (uint32_t w = lane; w < ix.S; w += 32) c += __popc(sM[r * ix.S + w]);
                        pc[r] = (r < R) ? __reduce_add_sync(FULL, c) : 0u;
                        if (r < R && pc[r] < pmin) {
                            pmin = pc[r];
                            rstar = r;
                        }
                    }
                    if (pmin == 0) alive = false;  // the group's AND emptied a table
                }
                if (alive) {
                    // A5 strategy (all give the same set): 1 dense scan of every ID,
                    // 2 sparse enumeration of rstar's hit cells, 3 union of the
                    // precomputed member bitmaps of the hit cells (or of the missed
                    // cells, complemented, when a table is mostly hit).  Auto picks
                    // the fewest warp-wide operations (Lemma 4.4's candidate term).
                    int stage = set_stage;
                    uint32_t list_total = 0;
#pragma unroll
                    for (int r = 0; r < RF; ++r)
                        if (r < R) list_total += pc[r] * 2 > ix.B ? ix.B - pc[r] : pc[r];
                    const bool union_ok = ix.mem_bits && list_total <= 2u * QK_ID_CAP;
                    if (stage == 3 && !union_ok) stage = 1;
                    if (stage == 0) {
                        const uint64_t kw = (ix.K + 31) / 32;
                        const uint64_t dense = kw * (uint64_t)(R + 2);
                        const uint64_t sparse = ((uint64_t)pmin * (ix.K / ix.B + 1) / 32 + pmin) * (uint64_t)(R + 3) + kw / 16;
                        uint64_t uni = ~0ull;
                        if (union_ok) {
                            uni = kw / 32 + 1;
#pragma unroll
                            for (int r = 0; r < RF; ++r) {
                                if (r >= R) continue;
                                const uint32_t cr = pc[r] < ix.B - pc[r] ? pc[r] : ix.B - pc[r];
                                uni += (uint64_t)cr * (kw / 32 + 1);
                            }
                        }
                        stage = (dense <= sparse && dense <= uni) ? 1 : (sparse <= uni ? 2 : 3);
                    }
                    if (leader) atomicAdd(&st->stage_count[stage], 1ull);
                    {
                        if (stage == 1) {
                            // dense: one ballot per 32 IDs becomes one bitmap word; four
                            // chunks per iteration so their table loads are in flight together
                            constexpr int DU = 4;
                            for (uint64_t i0 = (uint64_t)gw * 32 * DU; i0 < ix.K; i0 += (uint64_t)P * 32 * DU) {
                                uint32_t regw[DU];
                                uint4 ph[DU];
#pragma unroll
                                for (int u = 0; u < DU; ++u) {
                                    const uint64_t i = i0 + 32 * u + lane;
                                    regw[u] = i < ix.K ? __ldg(ix.reg + (i >> 5)) : 0u;
                                    ph[u] = i < ix.K ? __ldg(reinterpret_cast<const uint4*>(ix.phi) + i) : make_uint4(0, 0, 0, 0);
                                }
#pragma unroll
                                for (int u = 0; u < DU; ++u) {
                                    const uint64_t i = i0 + 32 * u + lane;
                                    bool ok = i < ix.K && ((regw[u] >> (i & 31)) & 1u);
                                    const uint32_t cell[8] = {ph[u].x & 0xffffu, ph[u].x >> 16, ph[u].y & 0xffffu,
                                                              ph[u].y >> 16,     ph[u].z & 0xffffu, ph[u].z >> 16,
                                                              ph[u].w & 0xffffu, ph[u].w >> 16};
#pragma unroll
                                    for (int r = 0; r < RF; ++r)
                                        if (r < R) ok &= (sM[r * ix.S + (cell[r] >> 5)] >> (cell[r] & 31)) & 1u;
                                    const unsigned bal = __ballot_sync(FULL, ok);
                                    if (lane == 0 && i0 + 32 * u < ix.K) sBits[(i0 >> 5) + u] = bal;
                                }
                            }
                        } else if (stage == 2) {
                            // sparse: the registered members of table rstar's hit cells,
                            // tested on the other tables.  Hit cells are taken one mask
                            // word (up to 32 cells) at a time; lane j holds cell j's
                            // member range, and the members of all those cells form one
                            // run of candidates, 128 per warp iteration (the group's
                            // warps interleave), whose IDs and partition rows are two
                            // independent coalesced loads.
                            const uint32_t* cellmask = sM + rstar * ix.S;
                            const uint64_t cbase = (uint64_t)rstar * ix.B;
                            // large cells (64+ members on average): one hit cell at a
                            // time, its members a contiguous run the group's warps share
                            const bool by_cell = ix.K >= 64ull * ix.B;
                            for (uint32_t w = 0; by_cell && w < ix.W; ++w) {
                                uint32_t hits = cellmask[w];
                                while (hits) {
                                    const uint64_t cell = cbase + w * 32 + (uint32_t)(__ffs(hits) - 1);
                                    hits &= hits - 1;
                                    const uint32_t m0 = (uint32_t)__ldg(ix.mem_off + cell);
                                    const uint32_t m1 = (uint32_t)__ldg(ix.mem_off + cell + 1);
                                    constexpr int SC = 4;
                                    for (uint32_t u0 = m0 + gw * 32 * SC; u0 < m1; u0 += P * 32 * SC) {
                                        uint32_t id[SC];
                                        uint4 ph[SC];
#pragma unroll
                                        for (int c = 0; c < SC; ++c) {
                                            const uint32_t pos = u0 + 32 * c + lane;
                                            const bool v = pos < m1;
                                            id[c] = v ? __ldg(ix.mem_ids + pos) : 0xffffffffu;
                                            ph[c] = v ? __ldg(ix.mem_phi + pos) : make_uint4(0, 0, 0, 0);
                                        }
#pragma unroll
                                        for (int c = 0; c < SC; ++c) {
                                            if (id[c] == 0xffffffffu) continue;
                                            const uint32_t cl[8] = {ph[c].x & 0xffffu, ph[c].x >> 16, ph[c].y & 0xffffu,
                                                                    ph[c].y >> 16,     ph[c].z & 0xffffu, ph[c].z >> 16,
                                                                    ph[c].w & 0xffffu, ph[c].w >> 16};
                                            bool ok = true;
#pragma unroll
                                            for (int r = 0; r < RF; ++r)
                                                if (r < R && r != rstar) ok &= (sM[r * ix.S + (cl[r] >> 5)] >> (cl[r] & 31)) & 1u;
                                            if (ok) atomicOr(sBits + (id[c] >> 5), 1u << (id[c] & 31));
                                        }
                                    }
                                }
                            }
                            for (uint32_t w = 0; !by_cell && w < ix.W; ++w) {
                                const uint32_t hits = cellmask[w];
                                if (!hits) continue;
                                uint32_t m0 = 0, cnt = 0;
                                if ((hits >> lane) & 1u) {
                                    const uint64_t cell = cbase + w * 32 + lane;
                                    m0 = (uint32_t)__ldg(ix.mem_off + cell);
                                    cnt = (uint32_t)__ldg(ix.mem_off + cell + 1) - m0;
                                }
                                uint32_t incl = cnt;
#pragma unroll
                                for (int off = 1; off < 32; off <<= 1) {
                                    const uint32_t y = __shfl_up_sync(FULL, incl, off);
                                    if (lane >= (unsigned)off) incl += y;
                                }
                                const uint32_t total = __shfl_sync(FULL, incl, 31);
                                const uint32_t base = m0 - (incl - cnt);  // list position of candidate u = base + u
                                constexpr int SU = 4;
                                for (uint32_t u0 = gw * 32 * SU; u0 < total; u0 += P * 32 * SU) {
                                    uint32_t id[SU];
                                    uint4 ph[SU];
#pragma unroll
                                    for (int c = 0; c < SU; ++c) {
                                        const uint32_t u = u0 + 32 * c + lane;
                                        // owner lane: the first lane whose inclusive count exceeds u
                                        uint32_t j = 0;
#pragma unroll
                                        for (uint32_t step = 16; step >= 1; step >>= 1) {
                                            const uint32_t e2 = __shfl_sync(FULL, incl, j + step - 1);
                                            if (e2 <= u) j += step;
                                        }
                                        const uint32_t pos = __shfl_sync(FULL, base, j) + u;
                                        const bool v = u < total;
                                        id[c] = v ? __ldg(ix.mem_ids + pos) : 0xffffffffu;
                                        ph[c] = v ? __ldg(ix.mem_phi + pos) : make_uint4(0, 0, 0, 0);
                                    }
#pragma unroll
                                    for (int c = 0; c < SU; ++c) {
                                        if (id[c] == 0xffffffffu) continue;
                                        const uint32_t cl[8] = {ph[c].x & 0xffffu, ph[c].x >> 16, ph[c].y & 0xffffu,
                                                                ph[c].y >> 16,     ph[c].z & 0xffffu, ph[c].z >> 16,
                                                                ph[c].w & 0xffffu, ph[c].w >> 16};
                                        bool ok = true;
#pragma unroll
                                        for (int r = 0; r < RF; ++r)
                                            if (r < R && r != rstar) ok &= (sM[r * ix.S + (cl[r] >> 5)] >> (cl[r] & 31)) & 1u;
                                        if (ok) atomicOr(sBits + (id[c] >> 5), 1u << (id[c] & 31));
                                    }
                                }
                            }
                        } else {
                            // union of member bitmaps: G_r = OR of the hit cells' bitmaps
                            // (or NOT of the missed cells' when over half are hit); the
                            // answer is registered AND every G_r.  Each warp lists the
                            // cells in its own staging words (warp prefix sums), then
                            // each lane ORs UW words per cell for UC cells at a time;
                            // the group's warps take interleaved word ranges.
                            uint16_t* list = reinterpret_cast<uint16_t*>(sIds);
                            uint32_t list_off[RF + 1];
                            list_off[0] = 0;
#pragma unroll
                            for (int r = 0; r < RF; ++r) {
                                uint32_t n_r = 0;
                                if (r < R) {
                                    const bool comp = pc[r] * 2 > ix.B;
                                    for (uint32_t c0 = 0; c0 < ix.W; c0 += 32) {
                                        const uint32_t cw = c0 + lane;
                                        uint32_t bits = 0;
                                        if (cw < ix.W) {
                                            bits = comp ? ~sM[r * ix.S + cw] : sM[r * ix.S + cw];
                                            if (cw == ix.W - 1 && (ix.B & 31)) bits &= (1u << (ix.B & 31)) - 1u;
                                        }
                                        const uint32_t c = __popc(bits);
                                        uint32_t incl = c;
#pragma unroll
                                        for (int off = 1; off < 32; off <<= 1) {
                                            const uint32_t y = __shfl_up_sync(FULL, incl, off);
                                            if (lane >= (unsigned)off) incl += y;
                                        }
                                        uint32_t pos = list_off[r] + n_r + incl - c;
                                        while (bits) {
                                            list[pos++] = (uint16_t)(cw * 32 + (__ffs(bits) - 1));
                                            bits &= bits - 1;
                                        }
                                        n_r += __shfl_sync(FULL, incl, 31);
                                    }
                                }
                                list_off[r + 1] = list_off[r] + n_r;
                            }
                            __syncwarp();
                            constexpr int UW = 4, UC = 4;
                            for (uint32_t wb = gw * 32 * UW; wb < bw; wb += P * 32 * UW) {
                                uint32_t g[UW];
#pragma unroll
                                for (int u = 0; u < UW; ++u) {
                                    const uint32_t w = wb + 32 * u + lane;
                                    g[u] = w < bw ? __ldg(ix.reg + w) : 0u;
                                }
#pragma unroll
                                for (int r = 0; r < RF; ++r) {
                                    if (r >= R) continue;
                                    const bool comp = pc[r] * 2 > ix.B;
                                    const uint32_t* mb = ix.mem_bits + (uint64_t)r * ix.B * bw;
                                    uint32_t acc[UW] = {0, 0, 0, 0};
                                    for (uint32_t t2 = list_off[r]; t2 < list_off[r + 1]; t2 += UC) {
                                        uint32_t v[UC][UW];
#pragma unroll
                                        for (int c = 0; c < UC; ++c) {
                                            const bool have = t2 + c < list_off[r + 1];
                                            const uint32_t* col = mb + (uint64_t)(have ? list[t2 + c] : 0) * bw;
#pragma unroll
                                            for (int u = 0; u < UW; ++u) {
                                                const uint32_t w = wb + 32 * u + lane;
                                                v[c][u] = (have && w < bw) ? __ldg(col + w) : 0u;
                                            }
                                        }
#pragma unroll
                                        for (int c = 0; c < UC; ++c)
#pragma unroll
                                            for (int u = 0; u < UW; ++u) acc[u] |= v[c][u];
                                    }
#pragma unroll
                                    for (int u = 0; u < UW; ++u) g[u] &= comp ? ~acc[u] : acc[u];
                                }
#pragma unroll
                                for (int u = 0; u < UW; ++u) {
                                    const uint32_t w = wb + 32 * u + lane;
                                    if (w < bw) sBits[w] = g[u];
                                }
                            }
                        }
                        qk_group_sync(P, gi);  // the bitmap is complete
                        // compaction: ascending IDs from the bitmap, bitmap cleared.
                        // Warp gw takes the gw-th contiguous run of 32-word blocks;
                        // 32 words (1024 IDs) at a time, lanes expand their word's
                        // bits into shared memory at their prefix position, then the
                        // warp copies the run out with coalesced stores.
                        const uint32_t nblk = (bw + 31) / 32;
                        const uint32_t wlo = (uint32_t)(((uint64_t)nblk * gw / P) * 32);
                        const uint32_t whi = min(bw, (uint32_t)(((uint64_t)nblk * (gw + 1) / P) * 32));
                        uint32_t mine_ids = 0;
                        for (uint32_t w = wlo + lane; w < whi; w += 32) mine_ids += __popc(sBits[w]);
                        mine_ids = __reduce_add_sync(FULL, mine_ids);
                        uint32_t before = 0;
                        if (lane == 0) ctl_cnt[gw] = mine_ids;
                        qk_group_sync(P, gi);
                        for (unsigned p2 = 0; p2 < P; ++p2) {
                            const uint32_t c2 = ctl_cnt[p2];
                            if (p2 < gw) before += c2;
                            count += c2;
                        }
                        // a dense answer is staged as the bitmap (fewer words)
                        const bool as_bits = count > o.bits_min && o.bits_words == bw;
                        const uint32_t words = as_bits ? bw : count;
                        if (leader) *ctl_start = count ? atomicAdd(&st->cursor, (unsigned long long)words) : 0ull;
                        qk_group_sync(P, gi);
                        start = *ctl_start;
                        const bool write = count && start + words <= o.stage_cap;
                        uint32_t at = before;
                        if (as_bits) {
                            for (uint32_t w = wlo + lane; w < whi; w += 32) {
                                if (write) o.stage[start + w] = sBits[w];
                                sBits[w] = 0;
                            }
                            start |= QSTART_BITMAP;
                        }
                        for (uint32_t w0b = wlo; w0b < whi && !as_bits; w0b += 32) {
                            const uint32_t w = w0b + lane;
                            uint32_t bits = (w < whi) ? sBits[w] : 0u;
                            uint32_t c = __popc(bits);
                            uint32_t incl = c;
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                uint32_t y = __shfl_up_sync(FULL, incl, off);
                                if (lane >= (unsigned)off) incl += y;
                            }
                            const uint32_t blk = __shfl_sync(FULL, incl, 31);
                            if (write && blk) {
                                uint32_t* dst = o.stage + start + at;
                                if (blk <= (uint32_t)QK_ID_CAP) {
                                    uint32_t pos = incl - c;
                                    while (bits) {
                                        sIds[pos++] = w * 32 + (__ffs(bits) - 1);
                                        bits &= bits - 1;
                                    }
                                    __syncwarp();
                                    for (uint32_t t2 = lane; t2 < blk; t2 += 32) dst[t2] = sIds[t2];
                                    __syncwarp();
                                } else {
                                    uint32_t pos = incl - c;
                                    while (bits) {
                                        dst[pos++] = w * 32 + (__ffs(bits) - 1);
                                        bits &= bits - 1;
                                    }
                                }
                            }
                            if (w < whi) sBits[w] = 0;
                            at += blk;
                        }
                        __syncwarp();
                    }
                }
                if (leader) {
                    o.qcount[q] = count;
                    o.qstart[q] = start;
                }
                qk_group_sync(P, gi);  // shared masks and control words are reused by the next query
            }
        }
        if (lane == 0 && probed) atomicAdd(&st->keys_probed, probed);
        if (lane == 0 && rows_read) atomicAdd(&st->rows_read, rows_read);
    }
}

}  // namespace rgb
