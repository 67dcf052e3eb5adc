// rambo_api.cu -- host side of the C ABI declared in include/rambo.h: handle
// life cycle, parameter derivation, input staging, kernel sequencing, status
// decoding and result hand-out.  Every step of insertion and query runs in the
// kernels of this library; the host only moves buffers and orders launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rambo_impl.cuh"

using namespace rgb;

namespace {

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RAMBO_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return RAMBO_ENOMEM;
    }
    return RAMBO_ECUDA;
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return map_cuda(e_); \
    } while (0)

#define RK(x)                    \
    do {                         \
        int r_ = (x);            \
        if (r_ != RAMBO_OK) return r_; \
    } while (0)

// growable device buffer (grown with 1/8 headroom, so batches of slightly
// varying size do not reallocate every call)
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
    int ensure(size_t n) {
        if (n <= cap && p) return RAMBO_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = n < 64 ? 64 : n + n / 8;
        if (cudaMalloc(&p, want * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return RAMBO_ENOMEM;
        }
        cap = want;
        return RAMBO_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// growable pinned host buffer (1/8 headroom, as DBuf: pinning is slow)
template <class T>
struct HBuf {
    T* p = nullptr;
    size_t cap = 0;
    int ensure(size_t n) {
        if (n <= cap && p) return RAMBO_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = n < 64 ? 64 : n + n / 8;
        if (cudaMallocHost(&p, want * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return RAMBO_ENOMEM;
        }
        cap = want;
        return RAMBO_OK;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

uint64_t splitmix_next(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    return mix64(state);
}

uint32_t stride_for(uint32_t W) {
    if (W <= 2) return W;
    if (W <= 4) return 4;
    return (W + 3) / 4 * 4;
}

// default build window: a slice of the index that stays resident in L2
constexpr uint64_t BUILD_TILE_BYTES = 128ull << 20;  // measured fastest on GB300 (L2 126 MB)

}  // namespace

struct rambo {
    uint64_t K = 0, m = 0, seed = 0;
    uint32_t B = 0, R = 0, eta = 0, L = 0, W = 0, S = 0;
    uint32_t B_local = 0, n_nodes = 1;  // two-level hash: B_local * n_nodes cells before any fold
    uint64_t tau_seed = 0, a_tau = 0, c_tau = 0;
    int device = 0, num_sms = 0;
    uint64_t a[RMAX] = {}, c[RMAX] = {};
    HashParams hp{};
    uint32_t* rows = nullptr;
    uint16_t* phi = nullptr;
    uint32_t* reg = nullptr;
    uint64_t* mem_off = nullptr;
    uint32_t* mem_ids = nullptr;
    uint4* mem_phi = nullptr;
    uint32_t* mem_bits = nullptr;
    DevStatus* st = nullptr;
    DevStatus* h_st = nullptr;  // pinned
    DevStatus* h_reset = nullptr;  // pinned: a clean status block, copied in before each query
    uint64_t* h_small = nullptr;  // pinned, 8 words
    // scratch
    DBuf<uint8_t> in_data;
    DBuf<uint64_t> in_off, in_ids, packed, qstart, scan_tmp, id_off;
    DBuf<uint32_t> stage, qcount, ids, fill, perm, chist, nmask;
    DBuf<uint64_t> ckeys, coff;
    DBuf<uint32_t> brec;               // bucketed build: update records
    DBuf<unsigned long long> bfill;    // bucketed build: per-window fill counters + overflow flag
    HBuf<uint32_t> h_ids;
    HBuf<uint64_t> h_id_off;
    // host-output pipeline: copy stream, per-chunk events, chunk bases and totals, status copies
    cudaStream_t cs = nullptr;
    cudaEvent_t pev[9] = {};
    DBuf<uint64_t> pslot;
    HBuf<uint64_t> ptot;
    HBuf<DevStatus> pst;
    rambo_query_config_t cfg{};
    uint64_t build_tile_bytes = BUILD_TILE_BYTES;
    int build_mode = 0;
    rambo_query_stats_t last{};
    uint64_t launches = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // call start, query start/end, call end
    uint64_t last_err_item = 0;
    // automatic block size: last (V, G, use_bitmap) resolved and its choice
    int auto_key = -1, auto_wpb = 0, auto_per_sm = 0;
    std::vector<rambo_plan_t*> plans;   // live plans (own or a server's) holding captured pointers
    unsigned char* na_base = nullptr;   // device address of the no-alloc query's fixed scratch

    IndexView view() const {
        IndexView v;
        v.rows = rows;
        v.m = m;
        v.R = R;
        v.eta = eta;
        v.shift = 64 - L;
        v.S = S;
        v.W = W;
        v.K = K;
        v.B = B;
        v.phi = phi;
        v.ps = phi_stride_for(R);
        v.reg = reg;
        v.mem_off = mem_off;
        v.mem_ids = mem_ids;
        v.mem_phi = mem_phi;
        v.mem_bits = mem_bits;
        return v;
    }
    uint64_t index_words() const { return (uint64_t)R * m * S; }
};

namespace {

void free_handle(rambo* h) {
    if (!h) return;
    for (rambo_plan_t* p : h->plans) plan_orphan(p);
    h->plans.clear();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->rows) cudaFree(h->rows);
    if (h->phi) cudaFree(h->phi);
    if (h->reg) cudaFree(h->reg);
    if (h->mem_off) cudaFree(h->mem_off);
    if (h->mem_ids) cudaFree(h->mem_ids);
    if (h->mem_phi) cudaFree(h->mem_phi);
    if (h->mem_bits) cudaFree(h->mem_bits);
    if (h->st) cudaFree(h->st);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->h_reset) cudaFreeHost(h->h_reset);
    if (h->h_small) cudaFreeHost(h->h_small);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    h->in_data.release();
    h->in_off.release();
    h->in_ids.release();
    h->packed.release();
    h->qstart.release();
    h->scan_tmp.release();
    h->id_off.release();
    h->stage.release();
    h->qcount.release();
    h->ids.release();
    h->fill.release();
    h->perm.release();
    h->chist.release();
    h->nmask.release();
    h->ckeys.release();
    h->brec.release();
    h->bfill.release();
    h->coff.release();
    h->h_ids.release();
    h->h_id_off.release();
    h->pslot.release();
    h->ptot.release();
    h->pst.release();
    for (auto& e : h->pev)
        if (e) cudaEventDestroy(e);
    if (h->cs) cudaStreamDestroy(h->cs);
    cudaSetDevice(cur);
    delete h;
}

// Member lists and member bitmaps of every cell (sparse and union set stages),
// rebuilt from the partition table; skipped when they would be too large.
// Rebuilds the registered members' lists in place (their buffers keep their
// addresses, so captured plans stay valid).  Needed whenever registration
// changes: inserts of new set IDs, merges, loads.
int refresh_cell_members(rambo* h, cudaStream_t s) {
    if (!h->mem_off) return RAMBO_OK;
    CK(launch_members(h->view(), h->mem_off, h->mem_ids, h->mem_phi, h->fill.p, s));
    return RAMBO_OK;
}

// Set-stage tables: per-cell member lists (registered sets only, with their
// partition rows) and per-cell member bitmaps.  Both serve only ID spaces a
// per-warp shared-memory bitmap can hold (K <= 4096 * 32).
int build_cell_members(rambo* h, cudaStream_t s) {
    if (h->mem_off) cudaFree(h->mem_off);
    if (h->mem_ids) cudaFree(h->mem_ids);
    if (h->mem_phi) cudaFree(h->mem_phi);
    if (h->mem_bits) cudaFree(h->mem_bits);
    h->mem_off = nullptr;
    h->mem_ids = nullptr;
    h->mem_phi = nullptr;
    h->mem_bits = nullptr;
    const uint64_t cells = (uint64_t)h->R * h->B, K = h->K;
    if ((K + 31) / 32 > 4096) return RAMBO_OK;
    if (cudaMalloc(&h->mem_off, (cells + 1 + scan_tmp_words(cells)) * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&h->mem_ids, (uint64_t)h->R * K * sizeof(uint32_t) + 16) != cudaSuccess ||
        cudaMalloc(&h->mem_phi, (uint64_t)h->R * K * sizeof(uint4) + 16) != cudaSuccess)
        return RAMBO_ENOMEM;
    RK(h->fill.ensure(cells));
    RK(refresh_cell_members(h, s));
    const uint64_t mb_bytes = cells * ((K + 31) / 32) * 4;
    if (mb_bytes <= (256ull << 20)) {
        if (cudaMalloc(&h->mem_bits, mb_bytes) != cudaSuccess) return RAMBO_ENOMEM;
        CK(launch_member_bits(h->view(), h->mem_bits, s));
    }
    return RAMBO_OK;
}

void default_config(rambo* h) {
    // One vector read per probe where the row allows it, as long as a lane's
    // words in flight (R * eta probes of V words each, all issued before any
    // is used) stay within 64 registers: wider tiles cost more in occupancy
    // than their fewer load instructions save.
    int V = 0, G = 0, fb_V = 0, fb_G = 0;
    for (int v = 4; v >= 1; v >>= 1) {
        if (h->S % (uint32_t)v) continue;
        int g = 1;
        while ((uint32_t)(g * v) < h->S) g *= 2;
        if (!query_config_supported(v, g, h->S)) continue;
        if (!fb_V) fb_V = v, fb_G = g;
        if (h->R * h->eta * (uint32_t)v <= 64) {
            V = v, G = g;
            break;
        }
    }
    if (!V) V = fb_V, G = fb_G;
    h->cfg.words_per_lane = (uint32_t)V;
    h->cfg.lanes_per_key = (uint32_t)G;
    h->cfg.warps_per_block = 0;  // chosen per call from the occupancy
    h->auto_key = -1;
    h->cfg.blocks_per_sm = 0;
    h->cfg.set_stage = 0;
    h->cfg.visit_order = 2;
    h->cfg.l2_fetch_bytes = 0;
    h->cfg.cluster = 0;
    // row reads through the read-only path with the L2 prefetch-size hint
    // .L2::64B: isolated rows then pull 64 B from DRAM instead of a 128-B
    // line; the random-read rate stays the same (it is bound by accesses,
    // not bytes), and the query kernels ran ~4% faster (uneven, genome)
    h->cfg.row_load = 7;
    h->cfg.warps_per_query = 0;
    h->cfg.host_chunks = 0;
    h->cfg.answer_staging = 0;
}

int decode_err(rambo* h, unsigned long long e) {
    if (e == NO_ERR) return RAMBO_OK;
    h->last_err_item = e >> 8;
    switch ((unsigned)(e & 0xff)) {
        case PRIO_ERANGE: return RAMBO_ERANGE;
        case PRIO_EINVAL: return RAMBO_EINVAL;
        case PRIO_EBADSEQ: return RAMBO_EBADSEQ;
        default: return RAMBO_ECUDA;
    }
}

// Staged view of a CSR batch on the device.  elem = bytes per data item.
int stage_batch(rambo* h, const void* data, size_t elem, const uint64_t* offsets, const uint64_t* set_ids,
                uint64_t n, int on_device, cudaStream_t s, BatchView& b, const void** d_data) {
    uint64_t off0, offN;
    if (on_device) {
        CK(cudaMemcpyAsync(h->h_small, offsets, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h->h_small + 1, offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        off0 = h->h_small[0];
        offN = h->h_small[1];
    } else {
        off0 = offsets[0];
        offN = offsets[n];
    }
    if (offN < off0) {
        h->last_err_item = 0;
        return RAMBO_EINVAL;
    }
    const uint64_t total = offN - off0;
    b.off0 = off0;
    b.total = total;
    b.n = n;
    if (on_device) {
        b.offsets = offsets;
        b.set_ids = set_ids;
        *d_data = static_cast<const uint8_t*>(data) + off0 * elem;
    } else {
        RK(h->in_off.ensure(n + 1));
        CK(cudaMemcpyAsync(h->in_off.p, offsets, (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        b.offsets = h->in_off.p;
        if (set_ids) {
            RK(h->in_ids.ensure(n));
            CK(cudaMemcpyAsync(h->in_ids.p, set_ids, n * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
            b.set_ids = h->in_ids.p;
        } else {
            b.set_ids = nullptr;
        }
        const uint8_t* src = static_cast<const uint8_t*>(data) + off0 * elem;
        // Bases in pinned host memory are read in place by the packing
        // kernel (one streaming pass over NVLink-C2C) instead of being copied
        // first; keys, small batches and pageable memory take the copy.
        cudaPointerAttributes pa{};
        if (elem == 1 && total >= (1u << 20) && cudaPointerGetAttributes(&pa, src) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer) {
            *d_data = pa.devicePointer;
        } else {
            cudaGetLastError();
            RK(h->in_data.ensure(total * elem + 16));
            if (total) CK(cudaMemcpyAsync(h->in_data.p, src, total * elem, cudaMemcpyHostToDevice, s));
            *d_data = h->in_data.p;
        }
    }
    return RAMBO_OK;
}

int pack_bases(rambo* h, BatchView& b, const void* d_bases, cudaStream_t s) {
    const uint64_t n_words = b.total / 32 + 2;  // one spare word for windows crossing the last word
    RK(h->packed.ensure(n_words));
    uint32_t* nmask = nullptr;
    if (b.skipn) {
        RK(h->nmask.ensure(n_words));
        nmask = h->nmask.p;
    }
    CK(launch_pack(static_cast<const uint8_t*>(d_bases), b.total, h->packed.p, n_words, h->st, s, nullptr, nmask));
    CK(launch_resolve_bad_base(b, h->st, s));
    b.packed = h->packed.p;
    b.nmask = nmask;
    return RAMBO_OK;
}

// Bucketed build of a validated, packed, registered batch: the input is cut
// into chunks whose update records (R*eta per key, 4 bytes each) fit a
// budget of device memory; per chunk one scatter launch files every record
// into its window's bucket (a chunk whose records overflow a bucket is filed
// again into larger ones) and one apply launch per window ORs the bucket
// into the rows.  Returns BUCKET_FALLBACK when memory or the bucket count
// does not allow it; the caller then builds window by window.
constexpr int BUCKET_FALLBACK = 1;
constexpr uint64_t BUCKET_WIN_BYTES = 48ull << 20;  // a window: well inside one die's share of L2

int insert_bucketed(rambo* h, const BatchView& b, cudaStream_t s) {
    const uint64_t rows_total = (uint64_t)h->R * h->m;
    // (48 MiB windows measured faster than 32 MiB ones of a power of two of
    // rows: genome 360 vs 485 ms, uneven 730 vs 866 ms)
    uint64_t rows_per_win = BUCKET_WIN_BYTES / ((uint64_t)h->S * 4);
    if (rows_per_win < 1) rows_per_win = 1;
    if (rows_per_win > rows_total) rows_per_win = rows_total;
    const uint64_t n_win64 = (rows_total + rows_per_win - 1) / rows_per_win;
    if (n_win64 > 4096) return BUCKET_FALLBACK;
    const uint32_t n_win = (uint32_t)n_win64;
    const uint64_t per_key = (uint64_t)h->R * h->eta;
    // records per chunk: up to 3e9 (12 GB), or a third of the free memory
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    uint64_t budget = (uint64_t)free_b / 3 / 4;
    if (budget > 3000000000ull) budget = 3000000000ull;
    if (budget < (1ull << 24)) return BUCKET_FALLBACK;
    uint64_t chunk_keys = (uint64_t)((double)budget / 1.6 / (double)per_key);
    if (chunk_keys > b.total) chunk_keys = b.total;
    if (chunk_keys < 1) chunk_keys = 1;
    // a window's share of a chunk's records (each distinct key's positions are
    // uniform over the rows; keys repeated across sets make the shares lumpier)
    const double expect = (double)chunk_keys * (double)per_key * (double)rows_per_win / (double)rows_total;
    uint64_t cap = (uint64_t)(expect * 1.5) + 65536;
    RK(h->bfill.ensure(n_win + 1));  // [n_win] fill counters, then the overflow flag
    const IndexView ix = h->view();
    for (uint64_t p_lo = 0; p_lo < b.total; p_lo += chunk_keys) {
        const uint64_t p_hi = p_lo + chunk_keys < b.total ? p_lo + chunk_keys : b.total;
        for (int attempt = 0;; ++attempt) {
            if (h->brec.ensure(n_win * cap) != RAMBO_OK) return BUCKET_FALLBACK;
            CK(cudaMemsetAsync(h->bfill.p, 0, (n_win + 1) * sizeof(unsigned long long), s));
            CK(launch_bucket_scatter(ix, h->hp, b, p_lo, p_hi, rows_per_win, n_win, cap, h->brec.p, h->bfill.p,
                                     h->bfill.p + n_win, h->st, h->num_sms, s));
            CK(cudaMemcpyAsync(h->h_small, h->bfill.p + n_win, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               s));
            CK(cudaStreamSynchronize(s));
            if (!h->h_small[0]) break;
            // a bucket overflowed: file the chunk again into larger buckets
            if (attempt == 3) return BUCKET_FALLBACK;
            cap *= 2;
        }
        for (uint32_t w = 0; w < n_win; ++w)
            CK(launch_bucket_apply(h->rows, (uint64_t)w * rows_per_win * h->S, h->brec.p, h->bfill.p, w, cap,
                                   h->num_sms, s));
    }
    return RAMBO_OK;
}

int run_insert(rambo* h, int seq, const uint64_t* set_ids, const void* data, const uint64_t* offsets,
               uint64_t n, uint32_t k, int on_device, cudaStream_t s) {
    if (!h || !offsets || !set_ids || (!data && n)) return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    if (seq && !split_k(k, &kk, &canon, &skipn)) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    CK(cudaSetDevice(h->device));
    BatchView b{};
    b.seq = seq;
    b.k = kk;
    b.canon = canon;
    b.skipn = skipn;
    const void* d_data = nullptr;
    RK(stage_batch(h, data, seq ? 1 : 8, offsets, set_ids, n, on_device, s, b, &d_data));
    CK(launch_status_reset(h->st, s));
    CK(launch_validate_batch(b, 0, h->K, h->st, s));
    if (seq) RK(pack_bases(h, b, d_data, s));
    else b.keys = static_cast<const uint64_t*>(d_data);
    CK(launch_register(b, h->reg, h->st, s));
    // Window by window (each an L2-sized slice of the rows) or one pass with
    // every atomic going to device memory, whichever the measured costs on
    // GB300 make cheaper: a window pass costs about 5 ps a key (extracting and
    // hashing it) plus about 4 us a launch; an atomic costs about 5 ps inside
    // a window and 40 ps as a device-memory read-modify-write.
    const uint64_t n_keys = b.total;  // upper bound for sequences
    const uint64_t rows_total = (uint64_t)h->R * h->m;
    uint64_t tile_rows = h->build_tile_bytes / ((uint64_t)h->S * 4);
    if (tile_rows < 1) tile_rows = 1;
    const uint64_t n_tiles = (rows_total + tile_rows - 1) / tile_rows;
    const double atomics = (double)h->R * h->eta;
    const double tiled_ps = (double)n_keys * ((double)n_tiles * 5.0 + atomics * 5.0) + (double)n_tiles * 4e6;
    const double untiled_ps = (double)n_keys * atomics * 40.0 + 4e6;
    const bool use_tiles = h->build_mode == 1 || (h->build_mode == 0 && n_tiles > 1 && tiled_ps < untiled_ps);
    // large builds: every key hashed once per input chunk, its updates filed
    // by window and applied window by window (k_build_bucket.cu)
    const bool bucket_ok = (uint64_t)h->R * h->eta <= 32;
    const bool use_buckets =
        bucket_ok && (h->build_mode == 3 ||
                      (h->build_mode == 0 && n_tiles > 1 && (double)n_keys * atomics >= (double)(1ull << 26)));
    if (use_buckets) {
        const int brc = insert_bucketed(h, b, s);
        if (brc != RAMBO_OK && brc != BUCKET_FALLBACK) return brc;
        if (brc == RAMBO_OK) goto built;
        // a bucket overflowed (keys far from uniform over the rows): build the
        // same bits window by window; the updates already applied are idempotent
    }
    if (use_tiles || use_buckets) {
        for (uint64_t lo = 0; lo < rows_total; lo += tile_rows) {
            uint64_t hi = lo + tile_rows < rows_total ? lo + tile_rows : rows_total;
            CK(launch_insert(h->view(), h->hp, b, lo, hi, h->st, h->num_sms, s));
        }
    } else {
        CK(launch_insert(h->view(), h->hp, b, 0, rows_total, h->st, h->num_sms, s));
    }
built:
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int rc = decode_err(h, h->h_st->err);
    if (rc == RAMBO_OK && h->h_st->spare[0]) {
        // new sets were registered: their cells' member lists change
        RK(refresh_cell_members(h, s));
        CK(cudaStreamSynchronize(s));
    }
    return rc;
}

struct QueryDest {
    int arena;              // 1: handle-owned arena
    uint32_t* ids;          // caller buffers (into variants)
    uint64_t ids_cap;
    uint64_t* id_offsets;
    uint64_t* needed;
    const uint32_t** out_ids;  // arena variants
    const uint64_t** out_off;
};

int resolve_tuning(rambo* h, uint64_t n, int& use_bitmap, QueryTuning& t) {
    t = QueryTuning{};
    if (query_is_wide(h->R, h->S)) {
        // rows wider than the register tiling or more than RF tables: one
        // thread block per query, as many resident as fit
        use_bitmap = 0;
        t.wide = 1;
        t.set_stage = 1;
        const int per_sm = query_wide_blocks_per_sm(h->R, h->S);
        if (per_sm < 1) return RAMBO_EINVAL;
        uint64_t blocks = (uint64_t)per_sm * h->num_sms;
        if (blocks > n) blocks = n;
        t.blocks = (int)(blocks < 1 ? 1 : blocks);
        t.warps_per_block = QW_THREADS / 32;
        t.batch = 1;
        return RAMBO_OK;
    }
    t.V = (int)h->cfg.words_per_lane;
    t.G = (int)h->cfg.lanes_per_key;
    t.warps_per_block = (int)h->cfg.warps_per_block;
    t.set_stage = (int)h->cfg.set_stage;
    t.order = (int)h->cfg.visit_order;
    t.load_kind = (int)h->cfg.row_load;
    t.staging = h->cfg.answer_staging;
    t.group = (int)h->cfg.warps_per_query;
    use_bitmap = (h->mem_off && t.set_stage != 1 && (h->K + 31) / 32 <= 4096) ? 1 : 0;
    const size_t spw_bytes = (size_t)query_smem_words_per_warp(h->R, h->S, h->K, use_bitmap) * 4;
    int per_sm = 0;
    if (t.warps_per_block == 0) {
        // The largest block that keeps at least 85% of the most warps any
        // block size can keep resident per SM.  The per-warp bitmap grows
        // with K, so for large ID spaces shared memory, not registers, limits
        // the residency and smaller blocks pack the SM more fully.
        const int key = (t.V * 64 + t.G) * 2 + use_bitmap;
        if (h->auto_key != key) {
            int nb_of[4] = {0, 0, 0, 0}, best = 0;
            for (int i = 0; i < 4; ++i) {
                const int w = 8 >> i;
                nb_of[i] = query_max_blocks_per_sm(t.V, t.G, h->eta, false, w, spw_bytes * (size_t)w);
                if (nb_of[i] * w > best) best = nb_of[i] * w;
            }
            if (best < 1) return RAMBO_EINVAL;
            for (int i = 0; i < 4; ++i)
                if (nb_of[i] > 0 && 100 * nb_of[i] * (8 >> i) >= 85 * best) {
                    h->auto_wpb = 8 >> i;
                    h->auto_per_sm = nb_of[i];
                    break;
                }
            h->auto_key = key;
        }
        t.warps_per_block = h->auto_wpb;
        per_sm = h->auto_per_sm;
    } else {
        per_sm = query_max_blocks_per_sm(t.V, t.G, h->eta, false, t.warps_per_block,
                                         spw_bytes * (size_t)t.warps_per_block);
    }
    if (per_sm < 1) return RAMBO_EINVAL;
    if (h->cfg.blocks_per_sm && (int)h->cfg.blocks_per_sm < per_sm) per_sm = (int)h->cfg.blocks_per_sm;
    uint64_t blocks = (uint64_t)per_sm * h->num_sms;
    uint64_t need = (n + t.warps_per_block - 1) / t.warps_per_block;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    t.blocks = (int)blocks;
    // grouped instance (several warps per query): up to one block a query
    t.blocks_group = 0;
    t.group_warps = 0;
    if (use_bitmap && t.group != 1 && t.warps_per_block > 1) {
        int per_sm_g = query_max_blocks_per_sm(t.V, t.G, h->eta, true, t.warps_per_block,
                                               query_group_smem_bytes(h->R, h->S, h->K, t.warps_per_block, t.group));
        if (h->cfg.blocks_per_sm && (int)h->cfg.blocks_per_sm < per_sm_g) per_sm_g = (int)h->cfg.blocks_per_sm;
        uint64_t bg = (uint64_t)per_sm_g * h->num_sms;
        if (bg > n) bg = n;
        if (bg >= 1) {
            t.blocks_group = (int)bg;
            t.group_warps = bg * (uint64_t)t.warps_per_block;
        }
    }
    uint64_t warps = blocks * t.warps_per_block;
    uint64_t batch = n / (warps * 32);
    if (batch < 1) batch = 1;
    if (batch > 16) batch = 16;
    t.batch = (int)batch;
    return RAMBO_OK;
}

// A clean status block (error words, work-queue ticket, cursor, counters)
// from the pinned template -- a copy, not a kernel -- then the intake:
// validation and 2-bit packing in one launch (the query kernel looks up the
// item of an unresolved base, if packing met one).  Sets the batch's packed,
// mask or key pointers.
int enqueue_intake(rambo* h, BatchView& b, const void* d_data, int seq, uint32_t k, cudaStream_t s) {
    CK(cudaMemcpyAsync(h->st, h->h_reset, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
    const uint8_t* bases = nullptr;
    uint64_t n_words = 0;
    b.nmask = nullptr;
    if (seq) {
        n_words = b.total / 32 + 2;  // one spare word for windows crossing the last word
        RK(h->packed.ensure(n_words));
        b.packed = h->packed.p;
        if (b.skipn) {
            RK(h->nmask.ensure(n_words));
            b.nmask = h->nmask.p;
        }
        bases = static_cast<const uint8_t*>(d_data);
    } else {
        b.keys = static_cast<const uint64_t*>(d_data);
    }
    CK(launch_intake(b, seq ? k : 1, h->K, bases, h->packed.p, n_words, const_cast<uint32_t*>(b.nmask), h->st, s));
    h->launches += 1;
    if (seq && b.skipn) {
        CK(launch_check_windows(b, h->st, s));
        h->launches += 1;
    }
    return RAMBO_OK;
}

// Host-output pipeline for large batches answered into the handle's pinned
// arena: the batch is cut into chunks of queries that run back to back on
// the call's stream (query kernel, count scan continuing from the previous
// chunk's total, gather), and each chunk's IDs and offsets go to pinned host
// memory on a second stream while the later chunks compute, so the
// device-to-host copy of the answers overlaps the query kernel instead of
// following it.  The device and pinned ID buffers and the staging arena
// must already be large enough (they are after a first call of that size);
// when the answers do not fit, it returns PIPE_FALLBACK with the staging
// arena grown, and the caller answers the batch the unpipelined way.
constexpr int PIPE_MAX_CHUNKS = 8;
constexpr uint64_t PIPE_MIN_QUERIES = 1u << 16;
constexpr int PIPE_FALLBACK = 1;

int run_query_pipelined(rambo* h, BatchView b, const void* d_data, int seq, uint32_t k, uint64_t n, cudaStream_t s,
                        QueryDest& d) {
    if (!h->ids.p || !h->h_ids.p || !h->stage.p) return PIPE_FALLBACK;
    if (!h->cs) CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
    for (auto& e : h->pev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    RK(h->pslot.ensure(PIPE_MAX_CHUNKS));
    RK(h->ptot.ensure(PIPE_MAX_CHUNKS));
    RK(h->pst.ensure(2));
    RK(h->id_off.ensure(n + 1));
    RK(h->h_id_off.ensure(n + 1));
    uint64_t* d_off = h->id_off.p;
    const uint64_t cap = h->ids.cap < h->h_ids.cap ? h->ids.cap : h->h_ids.cap;
    // 4 chunks measured best on the uneven workload (31.2 ms unchunked, 26.3 / 25.3 / 26.1 ms
    // with 2 / 4 / 8 chunks for 1e6 queries and 2.2 GB of answers)
    const int C = h->cfg.host_chunks ? (int)h->cfg.host_chunks : 4;
    uint64_t q_lo[PIPE_MAX_CHUNKS + 1];
    for (int c = 0; c <= C; ++c) q_lo[c] = n * (uint64_t)c / (uint64_t)C;

    CK(cudaEventRecord(h->ev[0], s));
    RK(enqueue_intake(h, b, d_data, seq, k, s));
    // the item holding an unresolved base, looked up over the whole batch
    // (the chunks' query kernels see only their slice)
    if (seq) {
        CK(launch_resolve_bad_base(b, h->st, s));
        h->launches += 1;
    }
    CK(cudaMemcpyAsync(h->pst.p, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->pev[PIPE_MAX_CHUNKS], s));
    CK(cudaMemsetAsync(h->pslot.p, 0, sizeof(uint64_t), s));
    CK(cudaEventRecord(h->ev[1], s));
    for (int c = 0; c < C; ++c) {
        const uint64_t nc = q_lo[c + 1] - q_lo[c];
        BatchView bc = b;
        bc.offsets = b.offsets + q_lo[c];
        bc.n = nc;
        bc.perm = nullptr;
        bc.no_resolve = 1;
        int ub = 0;
        QueryTuning t{};
        RK(resolve_tuning(h, nc, ub, t));
        QueryOut oc{h->stage.p, h->stage.cap, h->qstart.p + q_lo[c], h->qcount.p + q_lo[c], 0, 0};
        set_staging(oc, h->K, h->cfg.answer_staging);
        if (c) {  // fresh work queues for the chunk's query and gather kernels
            CK(cudaMemsetAsync(&h->st->ticket, 0, sizeof(unsigned long long), s));
            CK(cudaMemsetAsync(&h->st->gather_ticket, 0, sizeof(unsigned long long), s));
        }
        int nl = 0, n_scan = 0;
        CK(launch_query(h->view(), h->hp, bc, oc, t, ub, h->st, s, &nl));
        // chunk c's offsets continue from the total written by chunk c - 1's scan
        if (c) CK(cudaMemcpyAsync(h->pslot.p + c, d_off + q_lo[c], sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        CK(launch_scan_counts(oc.qcount, nc, d_off + q_lo[c], h->scan_tmp.p, h->scan_tmp.cap, s, nullptr, &n_scan,
                              h->pslot.p + c));
        CK(launch_gather(oc, d_off + q_lo[c], nc, h->ids.p, h->st, s, nullptr, cap));
        CK(cudaMemcpyAsync(h->ptot.p + c, d_off + q_lo[c + 1], sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(h->pev[c], s));
        h->launches += (uint64_t)(nl + n_scan + 1);
    }
    CK(cudaEventRecord(h->ev[2], s));
    CK(cudaMemcpyAsync(h->pst.p + 1, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->ev[3], s));
    // copies of each finished chunk, on the second stream
    CK(cudaEventSynchronize(h->pev[PIPE_MAX_CHUNKS]));
    const DevStatus in = h->pst.p[0];
    bool fits = in.err == NO_ERR && in.bad_pos == NO_ERR;
    uint64_t prev = 0;
    for (int c = 0; c < C && fits; ++c) {
        CK(cudaEventSynchronize(h->pev[c]));
        const uint64_t tot = h->ptot.p[c];
        if (tot < prev || tot > cap) {
            fits = false;
            break;
        }
        CK(cudaStreamWaitEvent(h->cs, h->pev[c], 0));
        if (tot > prev)
            CK(cudaMemcpyAsync(h->h_ids.p + prev, h->ids.p + prev, (tot - prev) * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, h->cs));
        const uint64_t o0 = c ? q_lo[c] + 1 : 0;
        CK(cudaMemcpyAsync(h->h_id_off.p + o0, d_off + o0, (q_lo[c + 1] + 1 - o0) * sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, h->cs));
        prev = tot;
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamSynchronize(h->cs));
    const DevStatus fin = h->pst.p[1];
    RK(decode_err(h, fin.err));
    if (!fits || fin.cursor > h->stage.cap) {
        RK(h->stage.ensure(fin.cursor));
        return PIPE_FALLBACK;
    }
    h->last.n_queries = n;
    h->last.keys_submitted = seq ? (b.total - n * (uint64_t)(k - 1)) : b.total;
    h->last.keys_probed = fin.keys_probed;
    h->last.rows_read = fin.rows_read;
    h->last.n_results = prev;
    for (int i = 0; i < 4; ++i) h->last.stage_queries[i] = fin.stage_count[i];
    h->last.staged_words = fin.cursor;
    // (the chunks' query kernels, interleaved with their scans and gathers)
    CK(cudaEventElapsedTime(&h->last.query_kernel_ms, h->ev[1], h->ev[2]));
    CK(cudaEventElapsedTime(&h->last.device_ms, h->ev[0], h->ev[3]));
    h->last.kernel_launches = h->launches;
    if (d.needed) *d.needed = prev;
    *d.out_ids = h->h_ids.p;
    *d.out_off = h->h_id_off.p;
    return RAMBO_OK;
}

int run_query(rambo* h, int seq, const void* data, const uint64_t* offsets, uint64_t n, uint32_t k,
              int on_device, cudaStream_t s, QueryDest& d) {
    if (!h || !offsets || (!data && n)) return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    if (seq && !split_k(k, &kk, &canon, &skipn)) return RAMBO_EINVAL;
    k = kk;
    CK(cudaSetDevice(h->device));
    h->last = rambo_query_stats_t{};
    h->launches = 0;
    if (n == 0) {
        if (d.arena) {
            if (on_device) {
                RK(h->id_off.ensure(1));
                CK(cudaMemsetAsync(h->id_off.p, 0, sizeof(uint64_t), s));
                CK(cudaStreamSynchronize(s));
                *d.out_off = h->id_off.p;
                *d.out_ids = reinterpret_cast<const uint32_t*>(h->ids.p);
            } else {
                RK(h->h_id_off.ensure(1));
                h->h_id_off.p[0] = 0;
                *d.out_off = h->h_id_off.p;
                *d.out_ids = h->h_ids.p;
            }
        } else if (on_device) {
            CK(cudaMemsetAsync(d.id_offsets, 0, sizeof(uint64_t), s));
            CK(cudaStreamSynchronize(s));
        } else {
            d.id_offsets[0] = 0;
        }
        if (d.needed) *d.needed = 0;
        return RAMBO_OK;
    }
    BatchView b{};
    b.seq = seq;
    b.k = k;
    b.canon = canon;
    b.skipn = skipn;
    const void* d_data = nullptr;
    RK(stage_batch(h, data, seq ? 1 : 8, offsets, nullptr, n, on_device, s, b, &d_data));
    int use_bitmap = 0;
    QueryTuning t{};
    RK(resolve_tuning(h, n, use_bitmap, t));
    RK(h->qcount.ensure(n));
    RK(h->qstart.ensure(n));
    RK(h->scan_tmp.ensure(scan_tmp_words(n)));
    if (h->stage.cap < (1u << 20)) RK(h->stage.ensure(1u << 20));
    if (!on_device && d.arena && n >= PIPE_MIN_QUERIES && !h->cfg.cluster && !h->cfg.l2_fetch_bytes &&
        h->cfg.host_chunks != 1) {
        const int rc = run_query_pipelined(h, b, d_data, seq, k, n, s, d);
        if (rc != PIPE_FALLBACK) return rc;
        h->launches = 0;
    }
    // device-side destination of the CSR offsets
    uint64_t* d_off;
    if (!d.arena && on_device) {
        d_off = d.id_offsets;
    } else {
        RK(h->id_off.ensure(n + 1));
        d_off = h->id_off.p;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        CK(cudaEventRecord(h->ev[0], s));
        RK(enqueue_intake(h, b, d_data, seq, k, s));
        b.perm = nullptr;
        if (h->cfg.cluster) {
            RK(h->ckeys.ensure(n));
            RK(h->perm.ensure(n));
            RK(h->chist.ensure(2 * CLUSTER_BUCKETS));
            RK(h->coff.ensure(CLUSTER_BUCKETS + 1));
            RK(h->scan_tmp.ensure(scan_tmp_words(n > CLUSTER_BUCKETS ? n : CLUSTER_BUCKETS)));
            CK(launch_cluster_order(b, h->ckeys.p, h->chist.p, h->coff.p, h->scan_tmp.p, h->scan_tmp.cap, h->perm.p,
                                    h->st, s));
            b.perm = h->perm.p;
            h->launches += 5;
        }
        QueryOut o{h->stage.p, h->stage.cap, h->qstart.p, h->qcount.p, 0, 0};
        set_staging(o, h->K, h->cfg.answer_staging);
        size_t l2_prev = 0;
        if (h->cfg.l2_fetch_bytes) {
            CK(cudaDeviceGetLimit(&l2_prev, cudaLimitMaxL2FetchGranularity));
            CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, h->cfg.l2_fetch_bytes));
        }
        CK(cudaEventRecord(h->ev[1], s));
        CK(launch_query(h->view(), h->hp, b, o, t, use_bitmap, h->st, s));
        CK(cudaEventRecord(h->ev[2], s));
        if (h->cfg.l2_fetch_bytes) CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, l2_prev));
        int n_scan = 0;
        CK(launch_scan_counts(h->qcount.p, n, d_off, h->scan_tmp.p, h->scan_tmp.cap, s, nullptr, &n_scan));
        h->launches += 1 + n_scan;
        CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h->h_small, d_off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        RK(decode_err(h, h->h_st->err));
        if (h->h_st->cursor <= h->stage.cap) break;
        if (attempt == 1) return RAMBO_ECUDA;  // the second run needs exactly the first's count
        RK(h->stage.ensure(h->h_st->cursor + (h->h_st->cursor >> 3)));
    }
    const uint64_t total_ids = h->h_small[0];
    h->last.n_queries = n;
    h->last.keys_submitted = seq ? (b.total - n * (uint64_t)(k - 1)) : b.total;
    h->last.keys_probed = h->h_st->keys_probed;
    h->last.rows_read = h->h_st->rows_read;
    h->last.n_results = total_ids;
    for (int i = 0; i < 4; ++i) h->last.stage_queries[i] = h->h_st->stage_count[i];
    h->last.staged_words = h->h_st->cursor;
    CK(cudaEventElapsedTime(&h->last.query_kernel_ms, h->ev[1], h->ev[2]));
    if (d.needed) *d.needed = total_ids;
    if (!d.arena && total_ids > d.ids_cap) return RAMBO_ENOSPC;
    QueryOut o{h->stage.p, h->stage.cap, h->qstart.p, h->qcount.p, 0, 0};
    set_staging(o, h->K, h->cfg.answer_staging);
    if (on_device) {
        uint32_t* d_ids;
        if (!d.arena) {
            d_ids = d.ids;
        } else {
            RK(h->ids.ensure(total_ids + 1));
            d_ids = h->ids.p;
        }
        CK(launch_gather(o, d_off, n, d_ids, h->st, s));
        CK(cudaEventRecord(h->ev[3], s));
        h->launches += 1;
        h->last.kernel_launches = h->launches;
        CK(cudaStreamSynchronize(s));
        CK(cudaEventElapsedTime(&h->last.device_ms, h->ev[0], h->ev[3]));
        if (d.arena) {
            *d.out_ids = d_ids;
            *d.out_off = d_off;
        }
        return RAMBO_OK;
    }
    uint32_t* hid;
    uint64_t* hoff;
    if (d.arena) {
        RK(h->h_ids.ensure(total_ids + 1));
        RK(h->h_id_off.ensure(n + 1));
        hid = h->h_ids.p;
        hoff = h->h_id_off.p;
    } else {
        hid = d.ids;
        hoff = d.id_offsets;
    }
    // (Gathering large answers straight into pinned host memory over
    // NVLink-C2C measured slower than gathering on the device and copying:
    // 1.9e6 against 2.15e6 keys/s end to end on the document workload.)
    RK(h->ids.ensure(total_ids + 1));
    uint32_t* d_ids = h->ids.p;
    CK(launch_gather(o, d_off, n, d_ids, h->st, s));
    CK(cudaEventRecord(h->ev[3], s));
    h->launches += 1;
    h->last.kernel_launches = h->launches;
    CK(cudaMemcpyAsync(hoff, d_off, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    if (total_ids) CK(cudaMemcpyAsync(hid, d_ids, total_ids * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaEventElapsedTime(&h->last.device_ms, h->ev[0], h->ev[3]));
    if (d.arena) {
        *d.out_ids = hid;
        *d.out_off = hoff;
    }
    return RAMBO_OK;
}

}  // namespace

namespace rgb {
// Read-only view of a handle for the fixed-scratch query entry point
// (rambo_noalloc.cu): index, hash parameters and the kernel tuning the handle
// would use for n queries.  Allocates nothing.
int handle_query_view(rambo_t* h, uint64_t n, IndexView* ix, HashParams* hp, QueryTuning* t, int* use_bitmap,
                      int* device) {
    if (!h || !ix || !hp || !t || !use_bitmap || !device) return RAMBO_EINVAL;
    RK(resolve_tuning(h, n, *use_bitmap, *t));
    *ix = h->view();
    *hp = h->hp;
    *device = h->device;
    return RAMBO_OK;
}

void handle_attach_plan(rambo_t* h, rambo_plan_t* p) {
    if (h) h->plans.push_back(p);
}

void handle_detach_plan(rambo_t* h, rambo_plan_t* p) {
    if (!h) return;
    for (size_t i = 0; i < h->plans.size(); ++i)
        if (h->plans[i] == p) {
            h->plans.erase(h->plans.begin() + (long)i);
            return;
        }
}

unsigned char* handle_noalloc_base(const rambo_t* h) { return h ? h->na_base : nullptr; }
}  // namespace rgb

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

static int create_impl(uint64_t K, uint32_t B_local, uint32_t n_nodes, uint32_t B, uint32_t R, uint64_t m, uint32_t eta,
                       uint64_t seed, uint64_t tau_seed, rambo_t** out) {
    if (!out) return RAMBO_EINVAL;
    *out = nullptr;
    if (K < 1 || K > (1ull << 32) || B < 1 || B > RAMBO_MAX_B || R < 1 || R > RAMBO_MAX_R || eta < 1 ||
        eta > RAMBO_MAX_ETA || m < 2 || m > (1ull << 32) || (m & (m - 1)) || B_local < 1 || n_nodes < 1 ||
        (uint64_t)B_local * n_nodes > 65535 || B > (uint64_t)B_local * n_nodes)
        return RAMBO_EINVAL;
    rambo* h = new (std::nothrow) rambo();
    if (!h) return RAMBO_ENOMEM;
    h->K = K;
    h->B = B;
    h->B_local = B_local;
    h->n_nodes = n_nodes;
    h->tau_seed = tau_seed;
    if (n_nodes > 1) {
        uint64_t ts = tau_seed;
        const uint64_t Pm = (1ull << 61) - 1;
        h->a_tau = 1 + splitmix_next(ts) % (Pm - 1);
        h->c_tau = splitmix_next(ts) % Pm;
    }
    h->R = R;
    h->m = m;
    h->eta = eta;
    h->seed = seed;
    while ((1ull << h->L) < m) ++h->L;
    h->W = (B + 31) / 32;
    h->S = stride_for(h->W);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return map_cuda(e);
    }
    // hash parameters, drawn from SplitMix64 in the specified order
    const uint64_t P = (1ull << 61) - 1;
    uint64_t state = seed;
    for (uint32_t r = 0; r < R; ++r) {
        h->a[r] = 1 + splitmix_next(state) % (P - 1);
        h->c[r] = splitmix_next(state) % P;
    }
    for (uint32_t r = 0; r < R; ++r)
        for (uint32_t j = 0; j < eta; ++j) h->hp.s[r][j] = splitmix_next(state) | 1ull;
    int rc = RAMBO_OK;
    auto fail = [&](int code) {
        free_handle(h);
        return code;
    };
    if (cudaMalloc(&h->rows, h->index_words() * 4) != cudaSuccess) return fail(RAMBO_ENOMEM);
    if (cudaMalloc(&h->phi, K * phi_stride_for(R) * sizeof(uint16_t)) != cudaSuccess) return fail(RAMBO_ENOMEM);
    if (cudaMalloc(&h->reg, ((K + 31) / 32) * 4) != cudaSuccess) return fail(RAMBO_ENOMEM);
    if (cudaMalloc(&h->st, sizeof(DevStatus)) != cudaSuccess) return fail(RAMBO_ENOMEM);
    if (cudaMallocHost(&h->h_st, sizeof(DevStatus)) != cudaSuccess) return fail(RAMBO_ENOMEM);
    if (cudaMallocHost(&h->h_reset, sizeof(DevStatus)) != cudaSuccess) return fail(RAMBO_ENOMEM);
    *h->h_reset = DevStatus{};
    h->h_reset->err = NO_ERR;
    h->h_reset->bad_pos = NO_ERR;
    if (cudaMallocHost(&h->h_small, 8 * sizeof(uint64_t)) != cudaSuccess) return fail(RAMBO_ENOMEM);
    for (auto& ev : h->ev)
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(RAMBO_ECUDA);
    cudaStream_t s = 0;
    if (cudaMemsetAsync(h->rows, 0, h->index_words() * 4, s) != cudaSuccess) return fail(RAMBO_ECUDA);
    if (cudaMemsetAsync(h->reg, 0, ((K + 31) / 32) * 4, s) != cudaSuccess) return fail(RAMBO_ECUDA);
    if (launch_phi_init(h->phi, K, R, B, h->a, h->c, h->B_local, h->n_nodes, h->a_tau, h->c_tau, s) != cudaSuccess)
        return fail(RAMBO_ECUDA);
    if (launch_status_reset(h->st, s) != cudaSuccess) return fail(RAMBO_ECUDA);
    rc = build_cell_members(h, s);
    if (rc) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(RAMBO_ECUDA);
    // the no-alloc query's scratch address and kernels, so that its calls
    // load and reserve nothing themselves
    rc = noalloc_setup(eta, &h->na_base);
    if (rc) return fail(rc);
    default_config(h);
    *out = h;
    return RAMBO_OK;
}

int rambo_create(uint64_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint64_t seed, rambo_t** out) {
    return create_impl(K, B, 1, B, R, m, eta, seed, 0, out);
}

int rambo_create_stacked(uint64_t K, uint32_t cells_per_node, uint32_t n_nodes, uint32_t R, uint64_t m, uint32_t eta,
                         uint64_t seed, uint64_t tau_seed, rambo_t** out) {
    if ((uint64_t)cells_per_node * n_nodes > RAMBO_MAX_B) return RAMBO_EINVAL;
    return create_impl(K, cells_per_node, n_nodes, cells_per_node * n_nodes, R, m, eta, seed, tau_seed, out);
}

uint32_t rambo_node_of(const rambo_t* h, uint64_t set_id) {
    if (!h || h->n_nodes <= 1) return 0;
    return (uint32_t)partition_hash(h->a_tau, h->c_tau, set_id, h->n_nodes);
}

int rambo_merge(rambo_t* dst, const rambo_t* src, void* stream) {
    if (!dst || !src || dst == src) return RAMBO_EINVAL;
    if (dst->K != src->K || dst->B != src->B || dst->R != src->R || dst->m != src->m || dst->eta != src->eta ||
        dst->seed != src->seed || dst->B_local != src->B_local || dst->n_nodes != src->n_nodes ||
        dst->tau_seed != src->tau_seed || dst->S != src->S || dst->device != src->device)
        return RAMBO_EINVAL;
    CK(cudaSetDevice(dst->device));
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_or_words(dst->rows, src->rows, dst->index_words(), s));
    CK(launch_or_words(dst->reg, src->reg, (dst->K + 31) / 32, s));
    RK(refresh_cell_members(dst, s));
    CK(cudaStreamSynchronize(s));
    return RAMBO_OK;
}

void rambo_destroy(rambo_t* h) { free_handle(h); }

int rambo_get_info(const rambo_t* h, rambo_info_t* out) {
    if (!h || !out) return RAMBO_EINVAL;
    out->K = h->K;
    out->B = h->B;
    out->R = h->R;
    out->eta = h->eta;
    out->L = h->L;
    out->m = h->m;
    out->seed = h->seed;
    out->row_words = h->W;
    out->row_stride = h->S;
    out->index_bytes = h->index_words() * 4;
    std::vector<uint32_t> regw((h->K + 31) / 32);
    if (cudaMemcpy(regw.data(), h->reg, regw.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return RAMBO_ECUDA;
    uint64_t n = 0;
    for (uint32_t w : regw) n += (uint64_t)__builtin_popcount(w);
    out->n_registered = n;
    out->nodes = h->n_nodes;
    out->cells_per_node = h->B_local;
    out->tau_seed = h->tau_seed;
    return RAMBO_OK;
}

int rambo_insert_batch(rambo_t* h, const uint64_t* set_ids, const uint64_t* keys, const uint64_t* offsets,
                       uint64_t n_sets, int on_device, void* stream) {
    return run_insert(h, 0, set_ids, keys, offsets, n_sets, 0, on_device, (cudaStream_t)stream);
}

int rambo_insert(rambo_t* h, uint64_t set_id, const uint64_t* keys, uint64_t n, int on_device, void* stream) {
    if (!h) return RAMBO_EINVAL;
    if (!on_device) {
        const uint64_t off[2] = {0, n};
        return run_insert(h, 0, &set_id, keys, off, 1, 0, 0, (cudaStream_t)stream);
    }
    // device keys: the set ID and offsets travel from the host, the keys stay on the device
    const uint64_t off[2] = {0, n};
    uint64_t* d = nullptr;
    CK(cudaSetDevice(h->device));
    if (cudaMalloc(&d, 3 * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        return RAMBO_ENOMEM;
    }
    const uint64_t host3[3] = {set_id, off[0], off[1]};
    cudaError_t e = cudaMemcpy(d, host3, sizeof(host3), cudaMemcpyHostToDevice);
    int rc = e == cudaSuccess ? run_insert(h, 0, d, keys, d + 1, 1, 0, 1, (cudaStream_t)stream) : map_cuda(e);
    cudaFree(d);
    return rc;
}

int rambo_suggest_params(uint64_t K, double n_mean, double V, double p, double delta, uint32_t* B, uint32_t* R,
                         uint64_t* m, uint32_t* eta) {
    if (!K || !(n_mean > 0) || !(V >= 1) || !(p > 0 && p < 1) || !(delta > 0 && delta < 1) || !B || !R || !m || !eta)
        return RAMBO_EINVAL;
    const double ln2 = 0.6931471805599453;
    // Lemma 4.4: E[q_t] = B R eta + (K/B)(V + Bp) R is smallest at B* = sqrt(K V / eta);
    // eta is not known yet, so take the optimal eta of a Bloom filter at rate p first
    double eta0 = std::log(1.0 / p) / ln2;
    if (eta0 < 1) eta0 = 1;
    if (eta0 > RAMBO_MAX_ETA) eta0 = RAMBO_MAX_ETA;
    double b = std::sqrt((double)K * V / eta0);
    uint32_t Bv = (uint32_t)std::llround(b);
    if (Bv < 2) Bv = 2;
    if (Bv > RAMBO_MAX_B) Bv = RAMBO_MAX_B;
    // Lemma 4.2: delta <= K (1 - (1-p)(1-1/B)^V)^R
    const double f = 1.0 - (1.0 - p) * std::pow(1.0 - 1.0 / Bv, V);
    uint32_t Rv = 0;
    for (uint32_t r = 1; r <= RAMBO_MAX_R; ++r)
        if ((double)K * std::pow(f, (double)r) <= delta) {
            Rv = r;
            break;
        }
    *B = Bv;
    // Bloom-filter size for n keys per cell at rate p: n ln(1/p) / (ln 2)^2
    const double n = n_mean * (double)K / Bv;
    const double mm = n * std::log(1.0 / p) / (ln2 * ln2);
    uint64_t mv = 2;
    while ((double)mv < mm && mv < (1ull << 32)) mv <<= 1;
    *m = mv;
    long e = std::lround(ln2 * (double)mv / n);
    if (e < 1) e = 1;
    if (e > RAMBO_MAX_ETA) e = RAMBO_MAX_ETA;
    *eta = (uint32_t)e;
    *R = Rv ? Rv : RAMBO_MAX_R;
    return Rv ? RAMBO_OK : RAMBO_ERANGE;
}

}  // extern "C"

namespace {

// Host k-mer keys of one sequence under the library's encoding (first base
// most significant; canonical = min with the reverse complement; skip-N =
// windows holding a byte outside ACGTacgt left out).  Returns RAMBO_EBADSEQ
// for such a byte without skip-N.
int host_kmers(const uint8_t* s, uint64_t n, uint32_t k, int canon, int skipn, std::vector<uint64_t>& out) {
    const uint64_t mask = k == 32 ? ~0ull : ((1ull << (2 * k)) - 1);
    uint64_t fwd = 0, rc = 0, run = 0;
    for (uint64_t p = 0; p < n; ++p) {
        const unsigned u = s[p] | 0x20u;
        int c = u == 'a' ? 0 : u == 'c' ? 1 : u == 'g' ? 2 : u == 't' ? 3 : -1;
        if (c < 0) {
            if (!skipn) return RAMBO_EBADSEQ;
            run = 0;
            c = 0;
        } else {
            ++run;
        }
        fwd = ((fwd << 2) | (uint64_t)c) & mask;
        rc = (rc >> 2) | ((uint64_t)(3 - c) << (2 * (k - 1)));
        if (p + 1 >= k && run >= k) out.push_back(canon && rc < fwd ? rc : fwd);
    }
    return RAMBO_OK;
}

}  // namespace

extern "C" {

int rambo_suggest_params_from_sample(uint64_t K, int kind, const void* data, const uint64_t* offsets,
                                     uint64_t n_sample, uint32_t k, double V, double p, double delta, uint32_t* B,
                                     uint32_t* R, uint64_t* m, uint32_t* eta, double* n_mean) {
    if (!offsets || !n_sample || (kind != 0 && kind != 1) || (!data && offsets[n_sample] > offsets[0]))
        return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    if (kind == 1 && !split_k(k, &kk, &canon, &skipn)) return RAMBO_EINVAL;
    // Sec. 5.1: the mean set cardinality, measured on the first sets of the
    // stream, sizes every BFU
    uint64_t distinct = 0;
    std::vector<uint64_t> keys;
    for (uint64_t t = 0; t < n_sample; ++t) {
        if (offsets[t + 1] < offsets[t]) return RAMBO_EINVAL;
        keys.clear();
        if (kind == 0) {
            const uint64_t* kp = static_cast<const uint64_t*>(data);
            keys.assign(kp + offsets[t], kp + offsets[t + 1]);
        } else {
            const int rc = host_kmers(static_cast<const uint8_t*>(data) + offsets[t], offsets[t + 1] - offsets[t], kk,
                                      canon, skipn, keys);
            if (rc) return rc;
        }
        std::sort(keys.begin(), keys.end());
        distinct += (uint64_t)(std::unique(keys.begin(), keys.end()) - keys.begin());
    }
    if (distinct == 0) return RAMBO_EINVAL;  // nothing to size the filters from
    const double mean = (double)distinct / (double)n_sample;
    if (n_mean) *n_mean = mean;
    return rambo_suggest_params(K, mean, V, p, delta, B, R, m, eta);
}

int rambo_insert_seq_batch(rambo_t* h, const uint64_t* set_ids, const uint8_t* bases, const uint64_t* offsets,
                           uint64_t n_sets, uint32_t k, int on_device, void* stream) {
    return run_insert(h, 1, set_ids, bases, offsets, n_sets, k, on_device, (cudaStream_t)stream);
}

int rambo_query_batch(rambo_t* h, const uint64_t* keys, const uint64_t* offsets, uint64_t n_queries, int on_device,
                      const uint32_t** ids, const uint64_t** id_offsets, void* stream) {
    if (!ids || !id_offsets) return RAMBO_EINVAL;
    QueryDest d{1, nullptr, 0, nullptr, nullptr, ids, id_offsets};
    return run_query(h, 0, keys, offsets, n_queries, 0, on_device, (cudaStream_t)stream, d);
}

int rambo_query_seq_batch(rambo_t* h, const uint8_t* bases, const uint64_t* offsets, uint64_t n_queries, uint32_t k,
                          int on_device, const uint32_t** ids, const uint64_t** id_offsets, void* stream) {
    if (!ids || !id_offsets) return RAMBO_EINVAL;
    QueryDest d{1, nullptr, 0, nullptr, nullptr, ids, id_offsets};
    return run_query(h, 1, bases, offsets, n_queries, k, on_device, (cudaStream_t)stream, d);
}

int rambo_query_batch_into(rambo_t* h, const uint64_t* keys, const uint64_t* offsets, uint64_t n_queries,
                           int on_device, uint32_t* ids, uint64_t ids_cap, uint64_t* id_offsets, uint64_t* needed,
                           void* stream) {
    if (!id_offsets || (!ids && ids_cap)) return RAMBO_EINVAL;
    QueryDest d{0, ids, ids_cap, id_offsets, needed, nullptr, nullptr};
    return run_query(h, 0, keys, offsets, n_queries, 0, on_device, (cudaStream_t)stream, d);
}

int rambo_query_seq_batch_into(rambo_t* h, const uint8_t* bases, const uint64_t* offsets, uint64_t n_queries,
                               uint32_t k, int on_device, uint32_t* ids, uint64_t ids_cap, uint64_t* id_offsets,
                               uint64_t* needed, void* stream) {
    if (!id_offsets || (!ids && ids_cap)) return RAMBO_EINVAL;
    QueryDest d{0, ids, ids_cap, id_offsets, needed, nullptr, nullptr};
    return run_query(h, 1, bases, offsets, n_queries, k, on_device, (cudaStream_t)stream, d);
}

int rambo_export_index(const rambo_t* h, uint32_t* host_words, uint64_t n_words) {
    if (!h || !host_words || n_words != h->index_words()) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy(host_words, h->rows, n_words * 4, cudaMemcpyDeviceToHost));
    return RAMBO_OK;
}

int rambo_export_registered(const rambo_t* h, uint32_t* host_words, uint64_t n_words) {
    if (!h || !host_words || n_words != (h->K + 31) / 32) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy(host_words, h->reg, n_words * 4, cudaMemcpyDeviceToHost));
    return RAMBO_OK;
}

int rambo_export_partition(const rambo_t* h, uint16_t* host_phi, uint64_t n) {
    if (!h || !host_phi || n != h->K * h->R) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    const uint32_t ps = phi_stride_for(h->R);
    std::vector<uint16_t> tmp(h->K * ps);
    CK(cudaMemcpy(tmp.data(), h->phi, tmp.size() * 2, cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < h->K; ++i)
        for (uint32_t r = 0; r < h->R; ++r) host_phi[i * h->R + r] = tmp[i * ps + r];
    return RAMBO_OK;
}

int rambo_cell_popcount(const rambo_t* h, uint64_t* host_out, void* stream) {
    if (!h || !host_out) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t cells = (uint64_t)h->R * h->B;
    unsigned long long* d = nullptr;
    CK(cudaMalloc(&d, cells * sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(d, 0, cells * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_cell_popcount(h->view(), d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, cells * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    return map_cuda(e);
}

int rambo_last_query_stats(const rambo_t* h, rambo_query_stats_t* out) {
    if (!h || !out) return RAMBO_EINVAL;
    *out = h->last;
    return RAMBO_OK;
}

int rambo_get_query_config(const rambo_t* h, rambo_query_config_t* out) {
    if (!h || !out) return RAMBO_EINVAL;
    *out = h->cfg;
    return RAMBO_OK;
}

int rambo_set_query_config(rambo_t* h, const rambo_query_config_t* cfg) {
    if (!h || !cfg) return RAMBO_EINVAL;
    // (indexes served by the block-per-query kernel ignore the tiling fields)
    if (!query_is_wide(h->R, h->S) && !query_config_supported((int)cfg->words_per_lane, (int)cfg->lanes_per_key, h->S))
        return RAMBO_EINVAL;
    if (cfg->warps_per_block != 0 && cfg->warps_per_block != 1 && cfg->warps_per_block != 2 &&
        cfg->warps_per_block != 4 && cfg->warps_per_block != 8)
        return RAMBO_EINVAL;
    if (cfg->set_stage > 3) return RAMBO_EINVAL;
    if (cfg->set_stage == 2 && !h->mem_off) return RAMBO_EINVAL;
    if (cfg->set_stage == 3 && !h->mem_bits) return RAMBO_EINVAL;
    if (cfg->visit_order > 2 || cfg->cluster > 1 || cfg->row_load > 7) return RAMBO_EINVAL;
    if (cfg->warps_per_query != 0 && cfg->warps_per_query != 1 && cfg->warps_per_query != 2 &&
        cfg->warps_per_query != 4 && cfg->warps_per_query != 8)
        return RAMBO_EINVAL;
    if (cfg->l2_fetch_bytes && cfg->l2_fetch_bytes != 32 && cfg->l2_fetch_bytes != 64 && cfg->l2_fetch_bytes != 128)
        return RAMBO_EINVAL;
    if (cfg->host_chunks > (uint32_t)PIPE_MAX_CHUNKS) return RAMBO_EINVAL;
    if (cfg->answer_staging > 64) return RAMBO_EINVAL;
    h->cfg = *cfg;
    return RAMBO_OK;
}

int rambo_list_query_configs(const rambo_t* h, rambo_query_config_t* out, int cap) {
    if (!h) return RAMBO_EINVAL;
    static const int vg[][2] = {{1, 1}, {2, 1}, {1, 2}, {4, 1}, {2, 2}, {4, 2}, {2, 4},
                                {4, 4}, {2, 8}, {1, 16}, {4, 8}, {4, 16}, {4, 32}};
    static const int wpb[] = {2, 4, 8};
    int n = 0;
    for (auto& p : vg) {
        if (!query_config_supported(p[0], p[1], h->S)) continue;
        for (int w : wpb) {
            if (out && n < cap) {
                out[n].words_per_lane = (uint32_t)p[0];
                out[n].lanes_per_key = (uint32_t)p[1];
                out[n].warps_per_block = (uint32_t)w;
                out[n].blocks_per_sm = 0;
                out[n].set_stage = 0;
                out[n].visit_order = 2;
                out[n].l2_fetch_bytes = 0;
                out[n].cluster = 0;
                out[n].row_load = h->cfg.row_load;
                out[n].warps_per_query = 0;
                out[n].host_chunks = h->cfg.host_chunks;
                out[n].answer_staging = h->cfg.answer_staging;
            }
            ++n;
        }
    }
    return n;
}

int rambo_query_one_per_launch(rambo_t* h, int kind, const void* data, const uint64_t* host_offsets,
                               uint64_t n_queries, uint32_t k, uint32_t* ids, uint32_t* counts, void* stream) {
    if (!h || !host_offsets || (!data && n_queries) || (n_queries && (!ids || !counts))) return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    if (kind == 1 && !split_k(k, &kk, &canon, &skipn)) return RAMBO_EINVAL;
    k = kk;
    if (kind != 0 && kind != 1) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    for (uint64_t q = 0; q < n_queries; ++q) {
        if (host_offsets[q + 1] < host_offsets[q]) return RAMBO_EINVAL;
        const uint64_t len = host_offsets[q + 1] - host_offsets[q];
        if (kind == 0 && len == 0) return RAMBO_EINVAL;
        if (kind == 1 && len < k) return RAMBO_EBADSEQ;
    }
    int* d_bad = reinterpret_cast<int*>(&h->st->spare[0]);
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    const IndexView ix = h->view();
    for (uint64_t q = 0; q < n_queries; ++q) {
        const uint64_t a = host_offsets[q], len = host_offsets[q + 1] - a;
        const uint8_t* bp = kind == 1 ? static_cast<const uint8_t*>(data) + a : nullptr;
        const uint64_t* kp = kind == 0 ? static_cast<const uint64_t*>(data) + a : nullptr;
        CK(launch_query_one(ix, h->hp, kind, bp, kp, len, k, canon, skipn, ids + q * h->K, counts + q, d_bad, s));
    }
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return bad ? RAMBO_EBADSEQ : RAMBO_OK;
}

int rambo_autotune(rambo_t* h, int kind, const void* data, const uint64_t* offsets, uint64_t n_queries, uint32_t k,
                   int on_device, int reps, rambo_query_config_t* best, void* stream) {
    if (!h || (kind != 0 && kind != 1) || reps < 1) return RAMBO_EINVAL;
    const int n = rambo_list_query_configs(h, nullptr, 0);
    std::vector<rambo_query_config_t> cands(n > 0 ? n : 1);
    rambo_list_query_configs(h, cands.data(), n);
    const rambo_query_config_t keep = h->cfg;
    rambo_query_config_t win = keep;
    float win_ms = -1.0f;
    // with the group size left automatic, pairs of warps sharing one query
    // (and its shared-memory bitmap) are tried too: on large ID spaces the
    // per-warp bitmap limits the queries in flight (document workload: 86.7
    // against 96.5 ms a batch)
    const uint32_t wpq_try[2] = {keep.warps_per_query, 2};
    const int n_wpq = (keep.warps_per_query == 0 && h->mem_off) ? 2 : 1;
    for (int c = 0; c < n; ++c) {
        for (int iw = 0; iw < n_wpq * 2; ++iw) {
            const uint32_t order = 1 + (uint32_t)(iw & 1);
            rambo_query_config_t cfg = cands[c];
            cfg.visit_order = order;
            cfg.set_stage = keep.set_stage;
            cfg.row_load = keep.row_load;
            cfg.warps_per_query = wpq_try[iw >> 1];
            cfg.host_chunks = keep.host_chunks;
            cfg.answer_staging = keep.answer_staging;
            if ((iw >> 1) && cfg.warps_per_block < 2) continue;
            if (rambo_set_query_config(h, &cfg) != RAMBO_OK) continue;
            float t_min = -1.0f;
            for (int r = 0; r < reps; ++r) {
                const uint32_t* ids = nullptr;
                const uint64_t* off = nullptr;
                int rc = kind == 0 ? rambo_query_batch(h, static_cast<const uint64_t*>(data), offsets, n_queries,
                                                       on_device, &ids, &off, stream)
                                   : rambo_query_seq_batch(h, static_cast<const uint8_t*>(data), offsets, n_queries, k,
                                                           on_device, &ids, &off, stream);
                if (rc) {
                    h->cfg = keep;
                    return rc;
                }
                if (t_min < 0 || h->last.device_ms < t_min) t_min = h->last.device_ms;
            }
            if (win_ms < 0 || t_min < win_ms) {
                win_ms = t_min;
                win = cfg;
            }
        }
    }
    h->cfg = win;
    if (best) *best = win;
    return RAMBO_OK;
}

int rambo_fold(rambo_t* h, void* stream) {
    if (!h || h->B < 2 || (h->B & 1)) return RAMBO_EINVAL;
    // folding frees and reallocates the rows and the set-stage tables that
    // a live plan's captured graph points to
    if (!h->plans.empty()) return RAMBO_ESTATE;
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t B2 = h->B / 2, W2 = (B2 + 31) / 32, S2 = stride_for(W2);
    const uint64_t n_rows = (uint64_t)h->R * h->m;
    uint32_t* rows2 = nullptr;
    if (cudaMalloc(&rows2, n_rows * S2 * 4) != cudaSuccess) {
        cudaGetLastError();
        return RAMBO_ENOMEM;
    }
    cudaError_t e = launch_fold(h->rows, n_rows, h->W, h->S, B2, W2, S2, rows2, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(rows2);
        return map_cuda(e);
    }
    cudaFree(h->rows);
    h->rows = rows2;
    h->B = B2;
    h->W = W2;
    h->S = S2;
    // a set's folded cell is its cell mod B/2 (cells b and b + B/2 merged)
    CK(launch_phi_init(h->phi, h->K, h->R, h->B, h->a, h->c, h->B_local, h->n_nodes, h->a_tau, h->c_tau, s));
    RK(build_cell_members(h, s));
    CK(cudaStreamSynchronize(s));
    default_config(h);
    return RAMBO_OK;
}

int rambo_set_build_tiling(rambo_t* h, uint64_t tile_bytes, int mode) {
    if (!h || mode < 0 || mode > 3) return RAMBO_EINVAL;
    if (tile_bytes) {
        if (tile_bytes < (uint64_t)h->S * 4) return RAMBO_EINVAL;
        h->build_tile_bytes = tile_bytes;
    }
    h->build_mode = mode;
    return RAMBO_OK;
}

int rambo_l2_fetch_granularity(uint32_t bytes, uint32_t* prev) {
    size_t v = 0;
    CK(cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity));
    if (prev) *prev = (uint32_t)v;
    if (bytes) {
        if (bytes != 32 && bytes != 64 && bytes != 128) return RAMBO_EINVAL;
        CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, bytes));
    }
    return RAMBO_OK;
}

uint64_t rambo_last_error_item(const rambo_t* h) { return h ? h->last_err_item : 0; }

// checkpoint: "RAMBOGB1", params, registered bitmap, rows
int rambo_save(const rambo_t* h, const char* path) {
    if (!h || !path) return RAMBO_EINVAL;
    CK(cudaSetDevice(h->device));
    FILE* f = fopen(path, "wb");
    if (!f) return RAMBO_EIO;
    uint64_t hdr[11] = {0x32424753424D4152ull, h->K, h->B, h->R, h->m, h->eta, h->seed, h->S,
                        h->B_local, h->n_nodes, h->tau_seed};
    bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1;
    std::vector<uint32_t> buf((h->K + 31) / 32);
    if (ok && cudaMemcpy(buf.data(), h->reg, buf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
    if (ok) ok = fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    const uint64_t chunk = 1ull << 24;  // words
    buf.resize(chunk);
    for (uint64_t w = 0; ok && w < h->index_words(); w += chunk) {
        uint64_t c = h->index_words() - w < chunk ? h->index_words() - w : chunk;
        if (cudaMemcpy(buf.data(), h->rows + w, c * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
        if (ok) ok = fwrite(buf.data(), 4, c, f) == c;
    }
    if (fclose(f) != 0) ok = false;
    return ok ? RAMBO_OK : RAMBO_EIO;
}

int rambo_load(const char* path, rambo_t** out) {
    if (!path || !out) return RAMBO_EINVAL;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return RAMBO_EIO;
    uint64_t hdr[11];
    if (fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 0x32424753424D4152ull) {
        fclose(f);
        return RAMBO_EINVAL;
    }
    rambo_t* h = nullptr;
    int rc = create_impl(hdr[1], (uint32_t)hdr[8], (uint32_t)hdr[9], (uint32_t)hdr[2], (uint32_t)hdr[3], hdr[4],
                         (uint32_t)hdr[5], hdr[6], hdr[10], &h);
    if (rc) {
        fclose(f);
        return rc;
    }
    if (h->S != hdr[7]) {
        fclose(f);
        rambo_destroy(h);
        return RAMBO_EINVAL;
    }
    bool ok = true;
    std::vector<uint32_t> buf((h->K + 31) / 32);
    ok = fread(buf.data(), 4, buf.size(), f) == buf.size();
    if (ok && cudaMemcpy(h->reg, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    const uint64_t chunk = 1ull << 24;
    buf.resize(chunk);
    for (uint64_t w = 0; ok && w < h->index_words(); w += chunk) {
        uint64_t c = h->index_words() - w < chunk ? h->index_words() - w : chunk;
        ok = fread(buf.data(), 4, c, f) == c;
        if (ok && cudaMemcpy(h->rows + w, buf.data(), c * 4, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    }
    fclose(f);
    if (!ok) {
        rambo_destroy(h);
        return RAMBO_EIO;
    }
    if (refresh_cell_members(h, nullptr) != RAMBO_OK || cudaStreamSynchronize(nullptr) != cudaSuccess) {
        rambo_destroy(h);
        return RAMBO_ECUDA;
    }
    *out = h;
    return RAMBO_OK;
}

int rambo_random_row_probe(const uint32_t* dev_buf, uint64_t n_rows, uint32_t row_words, uint64_t reads_per_thread,
                           uint32_t blocks, uint32_t threads, uint64_t seed, uint32_t row_load, float* ms,
                           void* stream) {
    if (!dev_buf || !ms || !blocks || !threads || threads > 256 || !n_rows)
        return RAMBO_EINVAL;
    if (!(row_words == 1 || row_words == 2 || row_words % 4 == 0) || row_load > 7) return RAMBO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaMalloc(&sink, 4));
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess)
        e = launch_random_rows(dev_buf, n_rows, row_words, reads_per_thread, seed, sink, (int)blocks, (int)threads,
                               (int)row_load, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return map_cuda(e);
}

const char* rambo_strerror(int code) {
    switch (code) {
        case RAMBO_OK: return "ok";
        case RAMBO_EINVAL: return "invalid argument";
        case RAMBO_ERANGE: return "set ID out of range";
        case RAMBO_EBADSEQ: return "bad sequence (byte outside ACGTacgt, or shorter than k)";
        case RAMBO_ENOMEM: return "out of memory";
        case RAMBO_ENOSPC: return "output buffer too small";
        case RAMBO_ECUDA: return "CUDA error";
        case RAMBO_ETIMEOUT: return "device wait timed out";
        case RAMBO_EIO: return "file I/O error";
        case RAMBO_ESTATE: return "invalid state";
        case RAMBO_E2BIG: return "request exceeds a fixed capacity (plan, server slot or no-allocation scratch)";
        default: return "unknown error";
    }
}

}  // extern "C"
