// k_util.cu -- small kernels around the RAMBO hot path: input validation and
// 2-bit packing (batch intake), set registration, the partition table and its
// per-cell member lists, the count scan and result gather of the compaction
// step, and index statistics.
#include "rambo_impl.cuh"

namespace rgb {

static inline int grid_for(uint64_t n, int threads, int cap = 1 << 20) {
    uint64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (uint64_t)cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------------------

__global__ void k_status_reset(DevStatus* st) {
    st->err = NO_ERR;
    st->bad_pos = NO_ERR;
    st->ticket = 0;
    st->cursor = 0;
    st->keys_probed = 0;
    st->rows_read = 0;
    st->spare[0] = st->spare[1] = 0;
    st->stage_count[0] = st->stage_count[1] = st->stage_count[2] = st->stage_count[3] = 0;
    st->gather_ticket = 0;
}

cudaError_t launch_status_reset(DevStatus* st, cudaStream_t s) {
    k_status_reset<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// partition table: phi[i*ps + r] = phi_r(i), ps = phi_stride_for(R) (8 or 16)

struct PhiParams {
    uint64_t a[RMAX], c[RMAX];
    uint64_t a_tau, c_tau;
    uint32_t B_local, n_nodes;
};

// cell of set i in table r: (B_local * tau(i) + phi_r(i)) mod B, phi_r over
// B_local cells, tau over n_nodes nodes (the two-level hash of the paper's
// node-parallel construction; one node gives the plain partition).  B is the
// current cell count, smaller than B_local * n_nodes after folding over.
__global__ void k_phi_init(uint16_t* phi, uint64_t K, uint32_t R, uint32_t B, PhiParams pp) {
    const uint32_t ps = phi_stride_for(R);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t node = pp.n_nodes > 1 ? partition_hash(pp.a_tau, pp.c_tau, i, pp.n_nodes) : 0;
        uint16_t row[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            uint64_t cell = 0;
            if (r < (int)R) cell = ((uint64_t)pp.B_local * node + partition_hash(pp.a[r], pp.c[r], i, pp.B_local)) % B;
            row[r] = (uint16_t)cell;
        }
#pragma unroll
        for (int h = 0; h < RMAX / 8; ++h) {
            if (h * 8u >= ps) break;
            uint4 v;
            v.x = row[8 * h + 0] | ((uint32_t)row[8 * h + 1] << 16);
            v.y = row[8 * h + 2] | ((uint32_t)row[8 * h + 3] << 16);
            v.z = row[8 * h + 4] | ((uint32_t)row[8 * h + 5] << 16);
            v.w = row[8 * h + 6] | ((uint32_t)row[8 * h + 7] << 16);
            reinterpret_cast<uint4*>(phi + i * ps)[h] = v;
        }
    }
}

cudaError_t launch_phi_init(uint16_t* phi, uint64_t K, uint32_t R, uint32_t B, const uint64_t* a, const uint64_t* c,
                            uint32_t B_local, uint32_t n_nodes, uint64_t a_tau, uint64_t c_tau, cudaStream_t s) {
    PhiParams pp{};
    for (uint32_t r = 0; r < R && r < (uint32_t)RMAX; ++r) {
        pp.a[r] = a[r];
        pp.c[r] = c[r];
    }
    pp.B_local = B_local;
    pp.n_nodes = n_nodes;
    pp.a_tau = a_tau;
    pp.c_tau = c_tau;
    k_phi_init<<<grid_for(K, 256, 4096), 256, 0, s>>>(phi, K, R, B, pp);
    return cudaGetLastError();
}

// OR of two indexes with identical layout (rows and registered bitmaps)
__global__ void k_or_words(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] |= src[i];
}

cudaError_t launch_or_words(uint32_t* dst, const uint32_t* src, uint64_t n, cudaStream_t s) {
    if (!n) return cudaSuccess;
    k_or_words<<<grid_for(n, 256, 152 * 64), 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batch validation: set IDs < K, non-decreasing offsets, minimum item length

// Validation of items [t0, n) with stride: set IDs < K, non-decreasing
// offsets, minimum length; a descriptor-driven batch must also start at 0
// and end exactly at the staged data's end.
__device__ __forceinline__ void validate_items(const BatchView& b, uint64_t min_len, unsigned short_prio, uint64_t K,
                                               DevStatus* st, uint64_t t0, uint64_t stride) {
    if (b.desc && t0 == 0 && (b.offsets[0] != 0 || b.offsets[b.n] != b.total)) record_error(st, 0, PRIO_EINVAL);
    for (uint64_t t = t0; t < b.n; t += stride) {
        if (b.set_ids && b.set_ids[t] >= K) {
            record_error(st, t, PRIO_ERANGE);
            continue;
        }
        uint64_t lo = b.offsets[t], hi = b.offsets[t + 1];
        if (hi < lo) {
            record_error(st, t, PRIO_EINVAL);
            continue;
        }
        if (hi - lo < min_len) record_error(st, t, short_prio);
    }
}

__global__ void k_validate(BatchView b, uint64_t min_len, unsigned short_prio, uint64_t K,
                           DevStatus* st) {
    bv_resolve(b);
    validate_items(b, min_len, short_prio, K, st, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
                   (uint64_t)gridDim.x * blockDim.x);
}

cudaError_t launch_validate_batch(const BatchView& b, uint64_t min_len, uint64_t K, DevStatus* st,
                                  cudaStream_t s) {
    if (b.n == 0 && !b.desc) return cudaSuccess;
    // a sequence query shorter than k is a bad sequence; an empty key query is invalid
    unsigned prio = b.seq ? PRIO_EBADSEQ : PRIO_EINVAL;
    k_validate<<<grid_for(b.n, 256, 8192), 256, 0, s>>>(b, min_len, prio, K, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2-bit packing of ASCII DNA: word w holds bases 32w..32w+31, base 32w+t in
// bits 63-2t..62-2t; A/a=0 C/c=1 G/g=2 T/t=3.  Bytes past the end pack as 0.
// A byte outside ACGTacgt is recorded (lowest position wins) and packs as 0.

__device__ __forceinline__ int base_code(unsigned ch) {
    unsigned u = ch | 0x20u;  // only 'A'/'a' etc. fold onto the lower-case letters
    bool ok = (u == 'a') | (u == 'c') | (u == 'g') | (u == 't');
    unsigned x = (u >> 1) & 3u;  // a->0, c->1, g->3, t->2
    return ok ? (int)(x ^ (x >> 1)) : -1;
}

// four ASCII bytes of a little-endian word -> the 2-bit code of each in the
// low bits of its byte (a->0 c->1 g->2 t->3; other bytes give some code)
__device__ __forceinline__ uint32_t codes4x(uint32_t w) {
    const uint32_t x = ((w | 0x20202020u) >> 1) & 0x03030303u;
    return x ^ ((x >> 1) & 0x01010101u);
}

// 0x80 in each byte of v that is zero, exactly (no borrow between bytes)
__device__ __forceinline__ uint32_t zero_bytes(uint32_t v) {
    return ~((((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v)) & 0x80808080u;
}

// 0x80 in each byte of a little-endian word that is one of ACGTacgt
__device__ __forceinline__ uint32_t acgt4(uint32_t w) {
    const uint32_t u = w | 0x20202020u;
    return zero_bytes(u ^ 0x61616161u) | zero_bytes(u ^ 0x63636363u) | zero_bytes(u ^ 0x67676767u) |
           zero_bytes(u ^ 0x74747474u);
}

// bytes flagged 0x80 (bits 7, 15, 23, 31) -> bits 0..3
__device__ __forceinline__ uint32_t unresolved_nibble(uint32_t m) {
    return (((m >> 7) * 0x00204081u) >> 21) & 0xfu;
}

// Packs words [w0, n_words) with stride.  With nmask (skip-N), bit t of
// nmask[w] marks base 32w + t as unresolved (packed as 0) and nothing is
// reported; bits past the end are 0.
__device__ __forceinline__ void pack_words(const uint8_t* __restrict__ bases, uint64_t total,
                                           uint64_t* __restrict__ packed, uint64_t n_words, DevStatus* st,
                                           uint32_t* __restrict__ nmask, uint64_t w0, uint64_t stride) {
    const bool aligned = (reinterpret_cast<uintptr_t>(bases) & 15) == 0;
    for (uint64_t w = w0; w < n_words; w += stride) {
        uint64_t v = 0;
        uint64_t p0 = w * 32;
        unsigned long long bad = NO_ERR;
        uint32_t um = 0;  // unresolved bases of this word
        if (aligned && p0 + 32 <= total) {
            // two 16-byte loads, four bases per 32-bit word, each word
            // handled as four bytes at once
            const uint4* q = reinterpret_cast<const uint4*>(bases + p0);
            const uint4 lo = __ldg(q), hi = __ldg(q + 1);
            const uint32_t wd[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t ok = acgt4(wd[i]);              // 0x80 in every byte that is a base
                const uint32_t badm = ~ok & 0x80808080u;       // 0x80 in every other byte
                if (badm) {
                    if (nmask) um |= unresolved_nibble(badm) << (4 * i);
                    else if (bad == NO_ERR) bad = p0 + 4 * i + ((__ffs(badm) - 1) >> 3);
                }
                const uint32_t c = codes4x(wd[i]) & ((ok >> 7) * 3u);  // an unresolved byte packs as 0
                // the four 2-bit codes, first base highest, into one byte
                v |= (uint64_t)((c * 0x40100401u) >> 24) << (56 - 8 * i);
            }
        } else {
            for (int t = 0; t < 32; ++t) {
                uint64_t p = p0 + t;
                if (p >= total) break;
                int c = base_code(__ldg(bases + p));
                if (c < 0) {
                    if (nmask) um |= 1u << t;
                    else if (bad == NO_ERR) bad = p;
                    c = 0;
                }
                v |= (uint64_t)c << (62 - 2 * t);
            }
        }
        packed[w] = v;
        if (nmask) nmask[w] = um;
        if (bad != NO_ERR) atomicMin(&st->bad_pos, bad);
    }
}

__global__ void k_pack(const uint8_t* __restrict__ bases, uint64_t total, uint64_t* __restrict__ packed,
                       uint64_t n_words, DevStatus* st, const uint64_t* __restrict__ desc,
                       uint32_t* __restrict__ nmask) {
    if (desc) {
        total = desc[1];
        n_words = total / 32 + 2;
    }
    pack_words(bases, total, packed, n_words, st, nmask, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
               (uint64_t)gridDim.x * blockDim.x);
}

// Query intake in one launch: validation of every query and, for DNA, the
// 2-bit packing of the batch (the two write only the error words and the
// packed buffers, so they need no ordering).  The item holding the lowest
// unresolved base is looked up by the query kernel (resolve_bad_base).
__global__ void k_intake(BatchView b, uint64_t min_len, unsigned short_prio, uint64_t K,
                         const uint8_t* __restrict__ bases, uint64_t* __restrict__ packed, uint64_t n_words,
                         uint32_t* __restrict__ nmask, DevStatus* st) {
    bv_resolve(b);
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    validate_items(b, min_len, short_prio, K, st, t0, stride);
    if (bases) pack_words(bases, b.total, packed, b.desc ? b.total / 32 + 2 : n_words, st, nmask, t0, stride);
}

cudaError_t launch_intake(const BatchView& b, uint64_t min_len, uint64_t K, const uint8_t* bases, uint64_t* packed,
                          uint64_t n_words, uint32_t* nmask, DevStatus* st, cudaStream_t s) {
    if (b.n == 0 && !b.desc) return cudaSuccess;
    const unsigned prio = b.seq ? PRIO_EBADSEQ : PRIO_EINVAL;
    const uint64_t work = b.n > n_words ? b.n : n_words;  // capacities for a descriptor batch
    k_intake<<<grid_for(work, 256, 1 << 16), 256, 0, s>>>(b, min_len, prio, K, bases, packed, n_words, nmask, st);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* bases, uint64_t total, uint64_t* packed, uint64_t n_words,
                        DevStatus* st, cudaStream_t s, const uint64_t* desc, uint32_t* nmask) {
    if (n_words == 0) return cudaSuccess;
    // with a descriptor, n_words is the capacity the grid is sized for
    k_pack<<<grid_for(n_words, 256, 1 << 16), 256, 0, s>>>(bases, total, packed, n_words, st, desc, nmask);
    return cudaGetLastError();
}

// Skip-N queries: query t needs k consecutive resolved bases somewhere in
// [a, e), i.e. a gap of at least k between consecutive unresolved bases (the
// range ends counting as unresolved).  Visits only the unresolved bits.
__global__ void k_check_windows(BatchView b, DevStatus* st) {
    bv_resolve(b);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < b.n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = b.offsets[t] - b.off0, e = b.offsets[t + 1] - b.off0;
        if (e < a + b.k) continue;  // decreasing or too short: reported by the validation
        uint64_t next = a;          // first base after the last unresolved one seen
        bool found = false;
        for (uint64_t w = a >> 5; w <= (e - 1) >> 5 && !found; ++w) {
            uint32_t x = b.nmask[w];
            if (w == (a >> 5)) x &= ~0u << (a & 31);
            if (w == ((e - 1) >> 5) && ((e - 1) & 31) != 31) x &= (2u << ((e - 1) & 31)) - 1u;
            while (x) {
                const uint64_t pos = w * 32 + (uint64_t)(__ffs(x) - 1);
                if (pos - next >= b.k) {
                    found = true;
                    break;
                }
                next = pos + 1;
                x &= x - 1;
            }
        }
        if (!found && e - next < b.k) record_error(st, t, PRIO_EBADSEQ);
    }
}

cudaError_t launch_check_windows(const BatchView& b, DevStatus* st, cudaStream_t s) {
    if (b.n == 0 && !b.desc) return cudaSuccess;
    k_check_windows<<<grid_for(b.n, 256, 8192), 256, 0, s>>>(b, st);
    return cudaGetLastError();
}

// The item holding the lowest bad byte gets an EBADSEQ error.
__global__ void k_resolve_bad_base(BatchView b, DevStatus* st) {
    bv_resolve(b);
    resolve_bad_base(b, st);
}

cudaError_t launch_resolve_bad_base(const BatchView& b, DevStatus* st, cudaStream_t s) {
    k_resolve_bad_base<<<1, 1, 0, s>>>(b, st);
    return cudaGetLastError();
}

// Every listed set ID becomes registered (Algorithm 2's SetIDs(M[b,r]) only
// reports inserted sets).  Runs only on a clean batch; counts the IDs that were
// not registered before in st->spare[0], so the host knows when the per-cell
// member lists need rebuilding.
__global__ void k_register(BatchView b, uint32_t* reg, DevStatus* st) {
    if (st->err != NO_ERR) return;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < b.n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t id = b.set_ids[t];
        const uint32_t bit = 1u << (id & 31);
        if (!(atomicOr(reg + (id >> 5), bit) & bit)) atomicAdd(&st->spare[0], 1ull);
    }
}

cudaError_t launch_register(const BatchView& b, uint32_t* reg, DevStatus* st, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    k_register<<<grid_for(b.n, 256, 4096), 256, 0, s>>>(b, reg, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 counts into uint64 offsets (n+1 entries, the last
// being the total).  Three passes: tile sums, scan of the tile sums, tiles.

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

uint64_t scan_tmp_words(uint64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* warp_tot,
                                                         uint64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        uint64_t u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(FULL, u, o);
            if (lane >= o) u += y;
        }
        warp_tot[lane] = u - t;  // exclusive prefix of warp totals
        if (lane == 31) *total = u;
    }
    __syncthreads();
    uint64_t r = warp_tot[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const uint32_t* __restrict__ counts, uint64_t n, uint64_t* __restrict__ out,
                             uint64_t* __restrict__ tile_sums, const uint64_t* __restrict__ n_dev,
                             const uint64_t* __restrict__ base_dev) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t tot;
    if (n_dev) n = *n_dev;
    const uint64_t base = base_dev ? *base_dev : 0;
    const uint64_t i0 = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t sum = 0;
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        v[t] = (i0 + t < n) ? counts[i0 + t] : 0;
        sum += v[t];
    }
    uint64_t pre = base + block_exclusive_scan(sum, warp_tot, &tot);
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        if (i0 + t < n) out[i0 + t] = pre;
        pre += v[t];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint64_t* tile_sums, uint64_t n_tiles, const uint64_t* __restrict__ n_dev) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t tot;
    if (n_dev) {
        const uint64_t n = *n_dev;
        n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
        if (n_tiles == 0) n_tiles = 1;
    }
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < n_tiles; b0 += blockDim.x) {
        uint64_t i = b0 + threadIdx.x;
        uint64_t v = i < n_tiles ? tile_sums[i] : 0;
        uint64_t pre = block_exclusive_scan(v, warp_tot, &tot);
        if (i < n_tiles) tile_sums[i] = carry + pre;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sums[n_tiles] = carry;
}

__global__ void k_scan_add(uint64_t* __restrict__ out, uint64_t n, const uint64_t* __restrict__ tile_sums,
                           uint64_t n_tiles, const uint64_t* __restrict__ n_dev, const uint64_t* __restrict__ base_dev,
                           unsigned long long* __restrict__ total_out) {
    if (n_dev) {
        n = *n_dev;
        n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
        if (n_tiles == 0) n_tiles = 1;
    }
    if ((uint64_t)blockIdx.x >= n_tiles) return;
    uint64_t add = tile_sums[blockIdx.x];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    for (int t = threadIdx.x; t < SCAN_TILE; t += blockDim.x)
        if (base + t < n) out[base + t] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[n] = tile_sums[n_tiles] + (base_dev ? *base_dev : 0);
        if (total_out) *total_out = out[n];
    }
}

// Small inputs: one block walks the tiles in order with a running carry (one
// launch instead of three; the batch's launch overhead, not the scan, is the
// cost there).
constexpr uint64_t SCAN_ONE_BLOCK_MAX = 8 * SCAN_TILE;

__global__ void k_scan_one_block(const uint32_t* __restrict__ counts, uint64_t n, uint64_t* __restrict__ out,
                                 const uint64_t* __restrict__ n_dev, const uint64_t* __restrict__ base_dev,
                                 unsigned long long* __restrict__ total_out) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t tot;
    if (n_dev) n = *n_dev;
    uint64_t carry = base_dev ? *base_dev : 0;
    for (uint64_t t0 = 0; t0 < n; t0 += SCAN_TILE) {
        const uint64_t base = t0 + (uint64_t)threadIdx.x * SCAN_ITEMS;
        uint64_t v[SCAN_ITEMS];
        uint64_t sum = 0;
#pragma unroll
        for (int t = 0; t < SCAN_ITEMS; ++t) {
            v[t] = (base + t < n) ? counts[base + t] : 0;
            sum += v[t];
        }
        uint64_t pre = carry + block_exclusive_scan(sum, warp_tot, &tot);
#pragma unroll
        for (int t = 0; t < SCAN_ITEMS; ++t) {
            if (base + t < n) out[base + t] = pre;
            pre += v[t];
        }
        carry += tot;  // read after the scan's closing barrier, rewritten only in the next tile's scan
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        if (total_out) *total_out = carry;
    }
}

cudaError_t launch_scan_counts(const uint32_t* counts, uint64_t n, uint64_t* offsets, uint64_t* tmp,
                               uint64_t tmp_words, cudaStream_t s, const uint64_t* n_dev, int* n_launched,
                               const uint64_t* base_dev, unsigned long long* total_out) {
    // with n_dev, n is the capacity the grids are sized for and the true count is read on the device;
    // with base_dev, every offset is shifted by the value it points to
    if (n <= SCAN_ONE_BLOCK_MAX) {
        k_scan_one_block<<<1, SCAN_THREADS, 0, s>>>(counts, n, offsets, n_dev, base_dev, total_out);
        if (n_launched) *n_launched = 1;
        return cudaGetLastError();
    }
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) tiles = 1;
    if (tmp_words < tiles + 1) return cudaErrorInvalidValue;
    k_scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(counts, n, offsets, tmp, n_dev, base_dev);
    k_scan_sums<<<1, SCAN_THREADS, 0, s>>>(tmp, tiles, n_dev);
    k_scan_add<<<(unsigned)tiles, 256, 0, s>>>(offsets, n, tmp, tiles, n_dev, base_dev, total_out);
    if (n_launched) *n_launched = 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// query clustering for cache locality: each query's locality key is the
// smallest hash over its terms (its minimizer); queries are bucketed by the
// key's top 16 bits, so queries sharing a minimizer (overlapping substrings
// of the same region) are handed out together and their common rows are read
// from L2.  Only the processing order changes; every query's answer is the same.

__global__ void k_minimizer(BatchView b, uint64_t* __restrict__ keys, uint32_t* __restrict__ hist,
                            const DevStatus* st) {
    if (st->err != NO_ERR) return;
    const int lane = threadIdx.x & 31;
    uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = warp; q < b.n; q += nwarps) {
        const uint64_t a = __ldg(b.offsets + q) - b.off0;
        const uint64_t e = __ldg(b.offsets + q + 1) - b.off0;
        const uint64_t nkeys = b.seq ? (e - a - b.k + 1) : (e - a);
        uint64_t mn = ~0ull;
        for (uint64_t t = lane; t < nkeys; t += 32) {
            uint64_t key = b.seq ? kmer_at(b.packed, a + t, b.k) : __ldg(b.keys + a + t);
            if (b.seq && b.canon) key = canonical_kmer(key, b.k);
            const uint64_t h = mix64(key ^ 0x5851F42D4C957F2Dull);
            mn = h < mn ? h : mn;
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const uint64_t o = __shfl_xor_sync(FULL, mn, off);
            mn = o < mn ? o : mn;
        }
        if (lane == 0) {
            keys[q] = mn;
            atomicAdd(hist + (mn >> 48), 1u);
        }
    }
}

__global__ void k_bucket_scatter(const uint64_t* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ off,
                                 uint32_t* __restrict__ fill, uint32_t* __restrict__ perm, const DevStatus* st) {
    if (st->err != NO_ERR) return;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t bk = (uint32_t)(keys[q] >> 48);
        perm[off[bk] + atomicAdd(fill + bk, 1u)] = (uint32_t)q;
    }
}

cudaError_t launch_cluster_order(const BatchView& b, uint64_t* keys, uint32_t* hist, uint64_t* bucket_off,
                                 uint64_t* scan_tmp, uint64_t scan_tmp_words, uint32_t* perm, const DevStatus* st,
                                 cudaStream_t s) {
    // hist holds 2 * CLUSTER_BUCKETS counters: counts, then fill cursors
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 2 * CLUSTER_BUCKETS, s);
    if (e != cudaSuccess) return e;
    if (b.n == 0) return cudaSuccess;
    k_minimizer<<<grid_for(b.n * 32, 256, 152 * 32), 256, 0, s>>>(b, keys, hist, st);
    e = launch_scan_counts(hist, CLUSTER_BUCKETS, bucket_off, scan_tmp, scan_tmp_words, s);
    if (e != cudaSuccess) return e;
    k_bucket_scatter<<<grid_for(b.n, 256, 4096), 256, 0, s>>>(keys, b.n, bucket_off, hist + CLUSTER_BUCKETS, perm, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gather staged result IDs into CSR order: one warp per query, warps taking
// GA_TAKE queries at a time from a work queue (answers range from nothing to
// the whole ID space, so a fixed share per warp would leave a long tail).  A
// query staged as its K-bit bitmap is expanded 32 words (up to 1024 IDs) at a
// time: every lane writes its word's set bits as IDs into the warp's run in
// shared memory at its prefix position, then the warp stores the run with
// coalesced writes (32 full words need no run: their IDs are consecutive).  The prefix of the lanes' bit counts (0..32, six bits)
// comes from six ballots, one per bit of the count, instead of a chain of
// shuffles.

constexpr int GA_THREADS = 256;
constexpr int GA_RUN = 1024;  // IDs of 32 bitmap words
constexpr int GA_RUN_PAD = GA_RUN + GA_RUN / 32;  // the run with one pad word per 32
constexpr unsigned GA_TAKE = 8;  // queries per work-queue ticket

__global__ void __launch_bounds__(GA_THREADS) k_gather(QueryOut o, const uint64_t* __restrict__ id_offsets, uint64_t n,
                                                        uint32_t* __restrict__ ids, DevStatus* st,
                                                        const uint64_t* __restrict__ n_dev, uint64_t ids_cap) {
    __shared__ uint32_t s_run[GA_THREADS / 32][GA_RUN_PAD];
    if (st->err != NO_ERR || st->cursor > o.stage_cap) return;
    if (n_dev) n = *n_dev;
    if (id_offsets[n] > ids_cap) return;  // the caller sees the total and reports the shortfall
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;  // lanes below this one
    uint32_t* run = s_run[threadIdx.x >> 5];
    for (;;) {
        unsigned long long q0 = 0;
        if (lane == 0) q0 = atomicAdd(&st->gather_ticket, (unsigned long long)GA_TAKE);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= n) break;
        const uint64_t q1 = min((unsigned long long)n, q0 + GA_TAKE);
        for (uint64_t q = q0; q < q1; ++q) {
            const uint32_t c = o.qcount[q];
            if (!c) continue;
            const uint64_t s0 = o.qstart[q];
            uint32_t* dst = ids + id_offsets[q];
            if (!(s0 & QSTART_BITMAP)) {
                // an ID list: four independent loads in flight per lane
                const uint32_t* src = o.stage + s0;
                uint32_t t = lane;
                for (; t + 96 < c; t += 128) {
                    const uint32_t a0 = __ldcs(src + t), a1 = __ldcs(src + t + 32);
                    const uint32_t a2 = __ldcs(src + t + 64), a3 = __ldcs(src + t + 96);
                    dst[t] = a0;
                    dst[t + 32] = a1;
                    dst[t + 64] = a2;
                    dst[t + 96] = a3;
                }
                for (; t < c; t += 32) dst[t] = __ldcs(src + t);
                continue;
            }
            // a bitmap, 32 words at a time; the words of the next two steps are
            // loaded ahead so their latency overlaps the expansion of this one
            const uint32_t* src = o.stage + (s0 & ~QSTART_BITMAP);
            const uint32_t bw = o.bits_words;
            uint32_t cur = lane < bw ? __ldcs(src + lane) : 0u;
            uint32_t nx1 = 32 + lane < bw ? __ldcs(src + 32 + lane) : 0u;
            uint32_t at = 0;
            for (uint32_t w0 = 0; w0 < bw; w0 += 32) {
                const uint32_t w = w0 + lane;
                const uint32_t nx2 = w + 64 < bw ? __ldcs(src + w + 64) : 0u;
                uint32_t bits = cur;
                cur = nx1;
                nx1 = nx2;
                const uint32_t cw = __popc(bits);
                uint32_t pos = 0, blk = 0;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const unsigned m = __ballot_sync(0xffffffffu, (cw >> k) & 1u);
                    pos += (uint32_t)__popc(m & lt) << k;
                    blk += (uint32_t)__popc(m) << k;
                }
                if (blk == GA_RUN) {
                    // 32 full words: the IDs are consecutive
                    for (uint32_t t = lane; t < GA_RUN; t += 32) dst[at + t] = w0 * 32 + t;
                    at += blk;
                    continue;
                }
                // the run is padded by one word per 32 (entry p at p + p/32), so
                // lanes whose words are full do not all write one bank
                if (blk > GA_RUN / 2) {
                    // dense words: every bit position in turn, no bit scans
#pragma unroll
                    for (int b = 0; b < 32; ++b) {
                        const uint32_t on = (bits >> b) & 1u;
                        if (on) run[pos + (pos >> 5)] = w * 32 + b;
                        pos += on;
                    }
                } else {
                    while (bits) {
                        run[pos + (pos >> 5)] = w * 32 + (__ffs(bits) - 1);
                        ++pos;
                        bits &= bits - 1;
                    }
                }
                __syncwarp();
                uint32_t t = lane;
                for (; t + 96 < blk; t += 128) {
                    const uint32_t a0 = run[t + (t >> 5)], a1 = run[t + 32 + ((t + 32) >> 5)];
                    const uint32_t a2 = run[t + 64 + ((t + 64) >> 5)], a3 = run[t + 96 + ((t + 96) >> 5)];
                    dst[at + t] = a0;
                    dst[at + t + 32] = a1;
                    dst[at + t + 64] = a2;
                    dst[at + t + 96] = a3;
                }
                for (; t < blk; t += 32) dst[at + t] = run[t + (t >> 5)];
                __syncwarp();  // the run is rewritten by the next 32 words
                at += blk;
            }
        }
    }
}

cudaError_t launch_gather(const QueryOut& o, const uint64_t* id_offsets, uint64_t n, uint32_t* ids,
                          DevStatus* st, cudaStream_t s, const uint64_t* n_dev, uint64_t ids_cap) {
    if (n == 0) return cudaSuccess;
    // one resident wave of warps serving the work queue
    static int wave[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !wave[dev]) {
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_gather),
                                                              GA_THREADS, 0);
        if (e != cudaSuccess) return e;
        wave[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int most = dev < 64 ? wave[dev] : 152 * 4;
    int blocks = grid_for(n * 32, GA_THREADS, most);
    k_gather<<<blocks, GA_THREADS, 0, s>>>(o, id_offsets, n, ids, st, n_dev, ids_cap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Loads the kernels of a sequence query other than the query kernel itself
// (status reset, validation, packing, bad-base lookup, scans, gather):
// cudaFuncGetAttributes makes the runtime load a kernel that lazy module
// loading would otherwise load at its first launch.

cudaError_t load_util_kernels() {
    const void* fns[] = {reinterpret_cast<const void*>(&k_status_reset), reinterpret_cast<const void*>(&k_validate),
                         reinterpret_cast<const void*>(&k_pack), reinterpret_cast<const void*>(&k_resolve_bad_base),
                         reinterpret_cast<const void*>(&k_scan_one_block), reinterpret_cast<const void*>(&k_scan_tiles),
                         reinterpret_cast<const void*>(&k_scan_sums), reinterpret_cast<const void*>(&k_scan_add),
                         reinterpret_cast<const void*>(&k_gather), reinterpret_cast<const void*>(&k_intake)};
    // (k_check_windows serves skip-N queries, which the no-alloc call does not take)
    for (const void* f : fns) {
        cudaFuncAttributes a;
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// folding over (appendix): cell b of the folded index is the OR of cells b and
// b + B/2.  Each thread rewrites whole rows from the old layout (W words,
// stride S) into the new one (W2 words, stride S2).

__device__ __forceinline__ uint32_t row_window(const uint32_t* row, uint32_t W, uint32_t x) {
    // the 32 bits starting at bit x of a row of W words (bits past the row are zero)
    const uint32_t wi = x >> 5, sh = x & 31;
    const uint32_t lo = wi < W ? row[wi] : 0u;
    if (!sh) return lo;
    const uint32_t hi = wi + 1 < W ? row[wi + 1] : 0u;
    return (lo >> sh) | (hi << (32 - sh));
}

__global__ void k_fold(const uint32_t* __restrict__ old_rows, uint64_t n_rows, uint32_t W, uint32_t S, uint32_t B2,
                       uint32_t W2, uint32_t S2, uint32_t* __restrict__ new_rows) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n_rows;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t* row = old_rows + p * S;
        uint32_t* out = new_rows + p * S2;
        for (uint32_t w = 0; w < S2; ++w) {
            uint32_t v = 0;
            if (w < W2) {
                v = row_window(row, W, 32 * w) | row_window(row, W, B2 + 32 * w);
                const uint32_t bits_here = B2 - 32 * w;  // cells of the folded row in this word
                if (bits_here < 32) v &= (1u << bits_here) - 1u;
            }
            out[w] = v;
        }
    }
}

cudaError_t launch_fold(const uint32_t* old_rows, uint64_t n_rows, uint32_t W, uint32_t S, uint32_t B2, uint32_t W2,
                        uint32_t S2, uint32_t* new_rows, cudaStream_t s) {
    k_fold<<<grid_for(n_rows, 256, 152 * 64), 256, 0, s>>>(old_rows, n_rows, W, S, B2, W2, S2, new_rows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// statistics: set bits of every Bloom filter (bit b of the rows of table r)

// Block (x, r, z) counts cells [z*CP_CELLS, (z+1)*CP_CELLS) of table r over
// its share of the rows, in shared-memory counters.
constexpr uint32_t CP_CELLS = 8192;

__global__ void k_cell_popcount(IndexView ix, unsigned long long* out) {
    __shared__ unsigned int cnt[CP_CELLS];
    const uint32_t r = blockIdx.y;
    const uint32_t c0 = blockIdx.z * CP_CELLS;
    const uint32_t nc = min(CP_CELLS, ix.B - c0);
    for (uint32_t b = threadIdx.x; b < nc; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const uint32_t* rows = ix.rows + (uint64_t)r * ix.m * ix.S;
    const uint32_t w_lo = c0 / 32, w_hi = (c0 + nc + 31) / 32;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < ix.m;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t* row = rows + p * ix.S;
        for (uint32_t w = w_lo; w < w_hi; ++w) {
            uint32_t x = row[w];
            while (x) {
                const uint32_t b = w * 32 + (uint32_t)(__ffs(x) - 1);
                atomicAdd(&cnt[b - c0], 1u);
                x &= x - 1;
            }
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nc; b += blockDim.x)
        if (cnt[b]) atomicAdd(out + (uint64_t)r * ix.B + c0 + b, (unsigned long long)cnt[b]);
}

cudaError_t launch_cell_popcount(const IndexView& ix, unsigned long long* out, cudaStream_t s) {
    dim3 grid((unsigned)grid_for(ix.m, 256, ix.B > CP_CELLS ? 128 : 512), ix.R, (ix.B + CP_CELLS - 1) / CP_CELLS);
    k_cell_popcount<<<grid, 256, 0, s>>>(ix, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-cell member lists of the registered sets (sparse set stage): counts,
// then placement of each ID with its partition row beside it, so the stage
// reads both with coalesced loads.  Order within a cell is arbitrary.
__global__ void k_member_count(const uint16_t* __restrict__ phi, const uint32_t* __restrict__ reg, uint64_t K,
                               uint32_t R, uint32_t B, uint32_t* __restrict__ cnt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (!((reg[i >> 5] >> (i & 31)) & 1u)) continue;
        for (uint32_t r = 0; r < R; ++r) atomicAdd(cnt + r * B + phi[i * phi_stride_for(R) + r], 1u);
    }
}

__global__ void k_member_place(const uint16_t* __restrict__ phi, const uint32_t* __restrict__ reg, uint64_t K,
                               uint32_t R, uint32_t B, const uint64_t* __restrict__ off, uint32_t* __restrict__ fill,
                               uint32_t* __restrict__ ids, uint4* __restrict__ rows) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (!((reg[i >> 5] >> (i & 31)) & 1u)) continue;
        // (the sparse stage's partition-row copy: the first 8 tables, all it reads)
        const uint4 row = reinterpret_cast<const uint4*>(phi + i * phi_stride_for(R))[0];
        for (uint32_t r = 0; r < R; ++r) {
            uint32_t cell = r * B + phi[i * phi_stride_for(R) + r];
            uint32_t at = atomicAdd(fill + cell, 1u);
            ids[off[cell] + at] = (uint32_t)i;
            rows[off[cell] + at] = row;
        }
    }
}

__global__ void k_member_bits(const uint16_t* __restrict__ phi, uint64_t K, uint32_t R, uint32_t B,
                              uint32_t* __restrict__ bits) {
    const uint64_t bw = (K + 31) / 32;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K;
         i += (uint64_t)gridDim.x * blockDim.x)
        for (uint32_t r = 0; r < R; ++r) {
            const uint64_t cell = (uint64_t)r * B + phi[i * phi_stride_for(R) + r];
            atomicOr(bits + cell * bw + (i >> 5), 1u << (i & 31));
        }
}

cudaError_t launch_member_bits(const IndexView& ix, uint32_t* mem_bits, cudaStream_t s) {
    const uint64_t words = (uint64_t)ix.R * ix.B * ((ix.K + 31) / 32);
    cudaError_t e = cudaMemsetAsync(mem_bits, 0, words * 4, s);
    if (e != cudaSuccess) return e;
    k_member_bits<<<grid_for(ix.K, 256, 4096), 256, 0, s>>>(ix.phi, ix.K, ix.R, ix.B, mem_bits);
    return cudaGetLastError();
}

cudaError_t launch_members(const IndexView& ix, uint64_t* mem_off, uint32_t* mem_ids, uint4* mem_phi,
                           uint32_t* fill, cudaStream_t s) {
    uint32_t cells = ix.R * ix.B;
    cudaError_t e = cudaMemsetAsync(fill, 0, sizeof(uint32_t) * cells, s);
    if (e != cudaSuccess) return e;
    k_member_count<<<grid_for(ix.K, 256, 4096), 256, 0, s>>>(ix.phi, ix.reg, ix.K, ix.R, ix.B, fill);
    // offsets from counts; tmp space: reuse the tail of mem_off (caller sized it)
    uint64_t* tmp = mem_off + cells + 1;
    e = launch_scan_counts(fill, cells, mem_off, tmp, scan_tmp_words(cells), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(fill, 0, sizeof(uint32_t) * cells, s);
    if (e != cudaSuccess) return e;
    k_member_place<<<grid_for(ix.K, 256, 4096), 256, 0, s>>>(ix.phi, ix.reg, ix.K, ix.R, ix.B, mem_off, fill,
                                                             mem_ids, mem_phi);
    return cudaGetLastError();
}

}  // namespace rgb
