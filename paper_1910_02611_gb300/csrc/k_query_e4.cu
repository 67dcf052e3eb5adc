// Query kernels for 3 <= eta <= 4 hashes per Bloom filter.
#define QK_ETA 4
#define QK_SUFFIX e4
#include "k_query_inst.cuh"
