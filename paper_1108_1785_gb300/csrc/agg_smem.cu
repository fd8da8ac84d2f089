// agg_smem.cu -- aggregation and key kernels for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_smem(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupSmem>(p, s, st);
}
cudaError_t launch_keys_smem(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupSmem>(p, s, keys, st);
}
}  // namespace gnm
