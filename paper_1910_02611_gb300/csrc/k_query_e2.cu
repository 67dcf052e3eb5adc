// Query kernels for eta <= 2 hashes per Bloom filter.
#define QK_ETA 2
#define QK_SUFFIX e2
#include "k_query_inst.cuh"
