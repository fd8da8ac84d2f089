// agg_l2.cu -- aggregation and key kernels for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_l2(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupL2>(p, s, st);
}
cudaError_t launch_keys_l2(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupL2>(p, s, keys, st);
}
}  // namespace gnm
