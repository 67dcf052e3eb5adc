// k_query_inst.cuh -- instantiates k_query<V, G, ETA> for one ETA (the
// including file defines QK_ETA and QK_SUFFIX) and exposes a launcher and the
// kernel addresses for occupancy queries.
#pragma once
#include "k_query.cuh"

// (words per lane V, lanes per key G) pairs the dispatcher knows
#define QK_VG_LIST(X) \
    X(1, 1) X(2, 1) X(1, 2) X(4, 1) X(2, 2) X(4, 2) X(2, 4) X(4, 4) X(2, 8) X(1, 16) X(4, 8) X(4, 16) X(4, 32)

#define QK_CAT2(a, b) a##b
#define QK_CAT(a, b) QK_CAT2(a, b)

namespace rgb {

const void* QK_CAT(qk_kernel_ptr_, QK_SUFFIX)(int V, int G, bool grouped) {
#define X(v, g)                                                                                   \
    if (V == v && G == g)                                                                         \
        return grouped ? reinterpret_cast<const void*>(&k_query<v, g, QK_ETA, true>)              \
                       : reinterpret_cast<const void*>(&k_query<v, g, QK_ETA, false>);
    QK_VG_LIST(X)
#undef X
    return nullptr;
}

cudaError_t QK_CAT(qk_launch_, QK_SUFFIX)(int V, int G, bool grouped, dim3 grid, dim3 block, size_t smem,
                                          cudaStream_t s, const IndexView& ix, const HashParams& hp,
                                          const BatchView& b, const QueryOut& o, int set_stage, int batch,
                                          uint32_t smem_per_warp, int use_bitmap, int order, int load_kind, int group,
                                          unsigned long long group_warps, DevStatus* st) {
#define X(v, g)                                                                                              \
    if (V == v && G == g) {                                                                                  \
        if (grouped)                                                                                         \
            k_query<v, g, QK_ETA, true><<<grid, block, smem, s>>>(ix, hp, b, o, set_stage, batch,            \
                                                                  smem_per_warp, use_bitmap, order,          \
                                                                  load_kind, group, group_warps, st);        \
        else                                                                                                 \
            k_query<v, g, QK_ETA, false><<<grid, block, smem, s>>>(ix, hp, b, o, set_stage, batch,           \
                                                                   smem_per_warp, use_bitmap, order,         \
                                                                   load_kind, group, group_warps, st);       \
        return cudaGetLastError();                                                                           \
    }
    QK_VG_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace rgb
