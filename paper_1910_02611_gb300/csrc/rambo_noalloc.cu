// rambo_noalloc.cu -- rambo_query_seq_batch_noalloc: the sequence query for
// callers that cannot allocate device memory while they query.
//
// It runs the same kernels as rambo_query_seq_batch_into, but every byte of
// working memory comes from one file-scope __device__ array instead of
// buffers the handle grows with cudaMalloc.  The call itself allocates
// nothing (no cudaMalloc, cudaFree or allocating library routine); it only
// launches kernels and copies a few words back to the stack.
//
// Set-up happens in rambo_create / rambo_load (which allocate anyway), with
// the handle's device current: cudaGetSymbolAddress gives the array's device
// address (under lazy module loading this is also when the array is
// reserved on that device), and every kernel the call can launch is loaded,
// so the first query does not load modules either.  The address is kept in
// the handle, so a handle created after a cudaDeviceReset holds the address
// of that new context.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; the status reset at the start of each call clears everything that
// must start at zero (error word, work-queue ticket, result cursor, counters),
// and all other regions are fully written before they are read.  Calls that
// overlap on the GPU race on the array.
#include "rambo_impl.cuh"

using namespace rgb;

namespace {

// limits of one call
constexpr uint64_t NA_MAX_QUERIES = 1ull << 19;
constexpr uint64_t NA_MAX_BASES = 1ull << 25;
constexpr uint64_t NA_STAGE_WORDS = 1ull << 22;

constexpr uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

// layout of the array (byte offsets, 256-byte aligned)
constexpr uint64_t NA_PACKED_WORDS = NA_MAX_BASES / 32 + 2;
constexpr uint64_t NA_SCAN_WORDS = NA_MAX_QUERIES / 4096 + 2;
constexpr uint64_t OFF_STATUS = 0;
constexpr uint64_t OFF_PACKED = align256(OFF_STATUS + sizeof(DevStatus));
constexpr uint64_t OFF_QCOUNT = align256(OFF_PACKED + NA_PACKED_WORDS * 8);
constexpr uint64_t OFF_QSTART = align256(OFF_QCOUNT + NA_MAX_QUERIES * 4);
constexpr uint64_t OFF_SCAN = align256(OFF_QSTART + NA_MAX_QUERIES * 8);
constexpr uint64_t OFF_STAGE = align256(OFF_SCAN + NA_SCAN_WORDS * 8);
constexpr uint64_t NA_SCRATCH_BYTES = align256(OFF_STAGE + NA_STAGE_WORDS * 4);
// the size the header states for the array
static_assert(sizeof(DevStatus) <= 256, "status block fits its 256-byte slot");
static_assert(NA_SCRATCH_BYTES == 31459072ull, "fixed scratch is the 31,459,072 bytes the header states");

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RAMBO_OK;
    return e == cudaErrorMemoryAllocation ? RAMBO_ENOMEM : RAMBO_ECUDA;
}

}  // namespace

// The fixed working memory.  In host code this name is a stand-in, not a
// device address: host code must use the address cudaGetSymbolAddress gives.
static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

namespace rgb {

int noalloc_setup(uint32_t eta, unsigned char** base) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return map_cuda(e == cudaSuccess ? cudaErrorUnknown : e);
    }
    e = load_util_kernels();
    if (e == cudaSuccess) e = load_query_kernels(eta);
    if (e == cudaSuccess) e = load_query_wide_kernel();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(e);
    }
    *base = static_cast<unsigned char*>(p);
    return RAMBO_OK;
}

}  // namespace rgb

namespace {

int decode(unsigned long long e) {
    if (e == NO_ERR) return RAMBO_OK;
    switch ((unsigned)(e & 0xff)) {
        case PRIO_ERANGE: return RAMBO_ERANGE;
        case PRIO_EINVAL: return RAMBO_EINVAL;
        case PRIO_EBADSEQ: return RAMBO_EBADSEQ;
        default: return RAMBO_ECUDA;
    }
}

#define NA_CK(x)                                       \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return map_cuda(e_);    \
    } while (0)

}  // namespace

extern "C" int rambo_query_seq_batch_noalloc(rambo_t* h, const uint8_t* bases, const uint64_t* offsets,
                                             uint64_t n_queries, uint32_t k, uint32_t* ids, uint64_t ids_cap,
                                             uint64_t* id_offsets, uint64_t* needed, void* stream) {
    if (!h || !offsets || !id_offsets || (!bases && n_queries) || (!ids && ids_cap)) return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    // skip-N windows need a per-base mask beyond the fixed array: not taken here
    if (!split_k(k, &kk, &canon, &skipn) || skipn) return RAMBO_EINVAL;
    k = kk;
    if (n_queries > NA_MAX_QUERIES) return RAMBO_E2BIG;
    const uint64_t n = n_queries;
    cudaStream_t s = (cudaStream_t)stream;
    IndexView ix;
    HashParams hp;
    QueryTuning t;
    int use_bitmap = 0, dev = 0;
    int rc = handle_query_view(h, n ? n : 1, &ix, &hp, &t, &use_bitmap, &dev);
    if (rc) return rc;
    NA_CK(cudaSetDevice(dev));
    unsigned char* base = handle_noalloc_base(h);
    if (!base) return RAMBO_ESTATE;
    if (n == 0) {
        NA_CK(cudaMemsetAsync(id_offsets, 0, sizeof(uint64_t), s));
        NA_CK(cudaStreamSynchronize(s));
        if (needed) *needed = 0;
        return RAMBO_OK;
    }
    uint64_t ends[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(&ends[0], offsets, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&ends[1], offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (ends[1] < ends[0]) return RAMBO_EINVAL;
    const uint64_t total = ends[1] - ends[0];
    if (total > NA_MAX_BASES) return RAMBO_E2BIG;

    DevStatus* st = reinterpret_cast<DevStatus*>(base + OFF_STATUS);
    uint64_t* packed = reinterpret_cast<uint64_t*>(base + OFF_PACKED);
    uint32_t* qcount = reinterpret_cast<uint32_t*>(base + OFF_QCOUNT);
    uint64_t* qstart = reinterpret_cast<uint64_t*>(base + OFF_QSTART);
    uint64_t* scan_tmp = reinterpret_cast<uint64_t*>(base + OFF_SCAN);
    uint32_t* stage = reinterpret_cast<uint32_t*>(base + OFF_STAGE);

    BatchView b{};
    b.seq = 1;
    b.offsets = offsets;
    b.off0 = ends[0];
    b.total = total;
    b.n = n;
    b.k = k;
    b.canon = canon;
    b.set_ids = nullptr;
    b.perm = nullptr;
    NA_CK(launch_status_reset(st, s));  // clears error word, ticket, cursor, counters
    b.packed = packed;
    // validation and packing in one launch (the query kernel reports an unresolved base)
    NA_CK(launch_intake(b, k, ix.K, bases + ends[0], packed, total / 32 + 2, nullptr, st, s));
    QueryOut o{stage, NA_STAGE_WORDS, qstart, qcount, 0, 0};
    set_staging(o, ix.K, t.staging);
    NA_CK(launch_query(ix, hp, b, o, t, use_bitmap, st, s));
    NA_CK(launch_scan_counts(qcount, n, id_offsets, scan_tmp, NA_SCAN_WORDS, s));
    DevStatus hst;
    uint64_t total_ids = 0;
    NA_CK(cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&total_ids, id_offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    rc = decode(hst.err);
    if (rc) return rc;
    if (hst.cursor > NA_STAGE_WORDS) return RAMBO_E2BIG;
    if (needed) *needed = total_ids;
    if (total_ids > ids_cap) return RAMBO_ENOSPC;
    NA_CK(launch_gather(o, id_offsets, n, ids, st, s));
    NA_CK(cudaStreamSynchronize(s));
    return RAMBO_OK;
}
