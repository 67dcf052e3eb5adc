// k_query.cu -- dispatch of the query kernel instances and occupancy helpers.
#include "k_query.cuh"

namespace rgb {

const void* qk_kernel_ptr_e2(int V, int G);
const void* qk_kernel_ptr_e4(int V, int G);
cudaError_t qk_launch_e2(int V, int G, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const IndexView& ix,
                         const HashParams& hp, const BatchView& b, const QueryOut& o, int set_stage, int batch,
                         uint32_t smem_per_warp, int use_bitmap, int order, int load_kind, DevStatus* st);
cudaError_t qk_launch_e4(int V, int G, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const IndexView& ix,
                         const HashParams& hp, const BatchView& b, const QueryOut& o, int set_stage, int batch,
                         uint32_t smem_per_warp, int use_bitmap, int order, int load_kind, DevStatus* st);

static const void* kernel_ptr(int V, int G, uint32_t eta) {
    return eta <= 2 ? qk_kernel_ptr_e2(V, G) : qk_kernel_ptr_e4(V, G);
}

bool query_config_supported(int V, int G, uint32_t S) {
    if (!qk_kernel_ptr_e2(V, G)) return false;
    if (S % (uint32_t)V) return false;
    uint32_t need = S / V;               // lanes needed to cover a row
    if ((uint32_t)G < need) return false;
    return (uint32_t)G < 2 * need || G == 1;  // at most half the lanes idle
}

uint32_t query_smem_words_per_warp(uint32_t R, uint32_t S, uint64_t K, int use_bitmap) {
    return R * S + QK_ID_CAP + (use_bitmap ? qk_bitmap_words(K) : 0);
}

int query_max_blocks_per_sm(int V, int G, uint32_t eta, int warps_per_block, size_t smem_per_block) {
    const void* f = kernel_ptr(V, G, eta);
    if (!f) return 0;
    if (smem_per_block > 48 * 1024)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_per_block) != cudaSuccess)
            return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, warps_per_block * 32, smem_per_block) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_query(const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                         const QueryTuning& t, int use_bitmap, DevStatus* st, cudaStream_t s) {
    if (b.n == 0 && !b.desc) return cudaSuccess;
    const uint32_t spw = query_smem_words_per_warp(ix.R, ix.S, ix.K, use_bitmap);
    const size_t smem = (size_t)spw * 4 * t.warps_per_block;
    const void* f = kernel_ptr(t.V, t.G, ix.eta);
    if (!f) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)t.blocks), block((unsigned)(t.warps_per_block * 32));
    if (ix.eta <= 2)
        return qk_launch_e2(t.V, t.G, grid, block, smem, s, ix, hp, b, o, t.set_stage, t.batch, spw, use_bitmap,
                            t.order, t.load_kind, st);
    return qk_launch_e4(t.V, t.G, grid, block, smem, s, ix, hp, b, o, t.set_stage, t.batch, spw, use_bitmap, t.order,
                        t.load_kind, st);
}

}  // namespace rgb
