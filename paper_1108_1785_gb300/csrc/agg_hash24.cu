// agg_hash24.cu -- aggregation and key kernels for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_hash24(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupHash24>(p, s, st);
}
cudaError_t launch_keys_hash24(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupHash24>(p, s, keys, st);
}
}  // namespace gnm
