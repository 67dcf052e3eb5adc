// k_query.cu -- dispatch of the query kernel instances and occupancy helpers.
#include "k_query.cuh"

namespace rgb {

const void* qk_kernel_ptr_e2(int V, int G, bool grouped);
const void* qk_kernel_ptr_e4(int V, int G, bool grouped);
cudaError_t qk_launch_e2(int V, int G, bool grouped, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                         int set_stage, int batch, uint32_t smem_per_warp, int use_bitmap, int order, int load_kind,
                         int group, unsigned long long group_warps, DevStatus* st);
cudaError_t qk_launch_e4(int V, int G, bool grouped, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                         int set_stage, int batch, uint32_t smem_per_warp, int use_bitmap, int order, int load_kind,
                         int group, unsigned long long group_warps, DevStatus* st);

static const void* kernel_ptr(int V, int G, uint32_t eta, bool grouped) {
    return eta <= 2 ? qk_kernel_ptr_e2(V, G, grouped) : qk_kernel_ptr_e4(V, G, grouped);
}

bool query_config_supported(int V, int G, uint32_t S) {
    if (!qk_kernel_ptr_e2(V, G, false)) return false;
    if (S % (uint32_t)V) return false;
    uint32_t need = S / V;               // lanes needed to cover a row
    if ((uint32_t)G < need) return false;
    return (uint32_t)G < 2 * need || G == 1;  // at most half the lanes idle
}

uint32_t query_smem_words_per_warp(uint32_t R, uint32_t S, uint64_t K, int use_bitmap) {
    // rounded to 16 bytes so every warp's control words stay 8-byte aligned
    return (QK_CTL + R * S + QK_ID_CAP + (use_bitmap ? qk_bitmap_words(K) : 0) + 3u) & ~3u;
}

// Shared memory of the grouped instance: every warp's control, mask and
// staging words, then one bitmap per query group.  group > 1 fixes the group
// size (min(group, warps per block)); group = 0 lets the device choose it
// from the batch, at least 2 warps, so a block holds at most wpb/2 groups.
size_t query_group_smem_bytes(uint32_t R, uint32_t S, uint64_t K, int wpb, int group) {
    const uint32_t small = query_smem_words_per_warp(R, S, K, 0);
    const uint32_t bwr = (qk_bitmap_words(K) + 3u) & ~3u;
    int P = group > 1 ? (group < wpb ? group : wpb) : 2;
    if (P < 2) P = 2;
    const int groups = wpb / P > 0 ? wpb / P : 1;
    return ((size_t)small * wpb + (size_t)bwr * groups) * 4;
}

int query_max_blocks_per_sm(int V, int G, uint32_t eta, bool grouped, int warps_per_block, size_t smem_per_block) {
    const void* f = kernel_ptr(V, G, eta, grouped);
    if (!f) return 0;
    if (smem_per_block > 48 * 1024)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_per_block) != cudaSuccess)
            return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, warps_per_block * 32, smem_per_block) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t load_query_kernels(uint32_t eta) {
    static const int vg[][2] = {{1, 1}, {2, 1}, {1, 2}, {4, 1}, {2, 2}, {4, 2}, {2, 4},
                                {4, 4}, {2, 8}, {1, 16}, {4, 8}, {4, 16}, {4, 32}};
    for (auto& p : vg)
        for (int grouped = 0; grouped < 2; ++grouped) {
            const void* f = kernel_ptr(p[0], p[1], eta, grouped != 0);
            if (!f) continue;
            cudaFuncAttributes a;
            const cudaError_t e = cudaFuncGetAttributes(&a, f);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

unsigned query_group_size(uint64_t n, int group, unsigned wpb, uint64_t group_warps, int use_bitmap) {
    return qk_group_size(n, group, wpb, group_warps, use_bitmap);
}

cudaError_t launch_query(const IndexView& ix, const HashParams& hp, const BatchView& b, const QueryOut& o,
                         const QueryTuning& t, int use_bitmap, DevStatus* st, cudaStream_t s, int* n_launched) {
    if (n_launched) *n_launched = 0;
    if (b.n == 0 && !b.desc) return cudaSuccess;
    if (t.wide) {
        const cudaError_t e = launch_query_wide(ix, hp, b, o, t.blocks, st, s);
        if (e == cudaSuccess && n_launched) *n_launched = 1;
        return e;
    }
    // one-warp instance: a bitmap in every warp's region; grouped instance:
    // one per group after the warps' regions
    const uint32_t spw_warp = query_smem_words_per_warp(ix.R, ix.S, ix.K, use_bitmap);
    const uint32_t spw_group = query_smem_words_per_warp(ix.R, ix.S, ix.K, 0);
    // Which instance serves the batch: known here for host-sized batches;
    // for a batch sized on the device (a captured plan) both are launched
    // and the one that does not match returns at once.
    bool run_warp = true, run_group = false;
    if (use_bitmap && t.group != 1 && t.blocks_group > 0) {
        if (b.desc) {
            run_group = true;
            run_warp = t.group == 0;
        } else {
            run_group = qk_group_size(b.n, t.group, (unsigned)t.warps_per_block, t.group_warps, use_bitmap) > 1;
            run_warp = !run_group;
        }
    }
    const dim3 block((unsigned)(t.warps_per_block * 32));
    for (int pass = 0; pass < 2; ++pass) {
        const bool grouped = pass == 1;
        if (grouped ? !run_group : !run_warp) continue;
        const void* f = kernel_ptr(t.V, t.G, ix.eta, grouped);
        if (!f) return cudaErrorInvalidValue;
        const uint32_t spw = grouped ? spw_group : spw_warp;
        const size_t smem = grouped ? query_group_smem_bytes(ix.R, ix.S, ix.K, t.warps_per_block, t.group)
                                    : (size_t)spw * 4 * t.warps_per_block;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const dim3 grid((unsigned)(grouped ? t.blocks_group : t.blocks));
        cudaError_t e = ix.eta <= 2
                            ? qk_launch_e2(t.V, t.G, grouped, grid, block, smem, s, ix, hp, b, o, t.set_stage, t.batch,
                                           spw, use_bitmap, t.order, t.load_kind, t.group, t.group_warps, st)
                            : qk_launch_e4(t.V, t.G, grouped, grid, block, smem, s, ix, hp, b, o, t.set_stage, t.batch,
                                           spw, use_bitmap, t.order, t.load_kind, t.group, t.group_warps, st);
        if (e != cudaSuccess) return e;
        if (n_launched) ++*n_launched;
    }
    return cudaSuccess;
}

}  // namespace rgb
