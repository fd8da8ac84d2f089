// agg_radix.cu -- aggregation and key kernels for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_radix(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupRadix>(p, s, st);
}
cudaError_t launch_keys_radix(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupRadix>(p, s, keys, st);
}
cudaError_t launch_keys_radixblk(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupRadixBlk>(p, s, keys, st);
}
cudaError_t launch_keys_radixblk2(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupRadixBlk2>(p, s, keys, st);
}
cudaError_t launch_keys_radixblk2h(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    return dev::launch_keys_impl<kLookupRadixBlk2H>(p, s, keys, st);
}
}  // namespace gnm
