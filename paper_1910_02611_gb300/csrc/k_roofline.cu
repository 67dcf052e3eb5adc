// k_roofline.cu -- random-row read microbenchmark: the achievable device-memory
// throughput for the access pattern of the query's row probes (independent
// random rows of row_words 32-bit words over a buffer the size of the index).
// It has no counterpart in the paper; it sets the denominator of the
// "fraction of the random-row roofline" the benchmark reports.
#include "rambo_impl.cuh"

namespace rgb {

template <int V>
__global__ void __launch_bounds__(256) k_random_rows(const uint32_t* __restrict__ buf, uint64_t n_rows,
                                                     uint32_t stride, uint64_t reads_per_thread, uint64_t seed,
                                                     int load_kind, uint32_t* sink) {
    constexpr int U = 16;  // independent reads in flight per thread
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t ctr = seed ^ (tid * 0x9E3779B97F4A7C15ull);
    uint32_t acc = 0;
    for (uint64_t it = 0; it < reads_per_thread; it += U) {
        uint32_t v[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t row = __umul64hi(mix64(ctr + u), n_rows);  // uniform in [0, n_rows)
            const uint32_t* p = buf + row * stride;
            if constexpr (V == 1) {
                v[u][0] = ld_row1(p, load_kind);
            } else if constexpr (V == 2) {
                uint2 t = ld_row2(p, load_kind);
                v[u][0] = t.x;
                v[u][1] = t.y;
            } else {
                uint4 t = ld_row4(p, load_kind);
                v[u][0] = t.x;
                v[u][1] = t.y;
                v[u][2] = t.z;
                v[u][3] = t.w;
            }
        }
        ctr += U;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int w = 0; w < V; ++w) acc ^= v[u][w];
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads alive
}

cudaError_t launch_random_rows(const uint32_t* buf, uint64_t n_rows, uint32_t row_words, uint64_t reads_per_thread,
                               uint64_t seed, uint32_t* sink, int blocks, int threads, int load_kind, cudaStream_t s) {
    if (n_rows == 0) return cudaErrorInvalidValue;
    const uint64_t rows = n_rows;
    if (row_words == 1)
        k_random_rows<1><<<blocks, threads, 0, s>>>(buf, rows, 1, reads_per_thread, seed, load_kind, sink);
    else if (row_words == 2)
        k_random_rows<2><<<blocks, threads, 0, s>>>(buf, rows, 2, reads_per_thread, seed, load_kind, sink);
    else if (row_words % 4 == 0)
        k_random_rows<4><<<blocks, threads, 0, s>>>(buf, rows, row_words, reads_per_thread, seed, load_kind, sink);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace rgb
