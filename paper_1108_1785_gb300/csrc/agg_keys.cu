// agg_keys.cu -- aggregation kernels of split launches: per-record keys precomputed by a
// lookup kernel (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_keys(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupKeys>(p, s, st);
}
}  // namespace gnm
