// agg_radix.cu -- aggregation kernel variants for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_radix(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupRadix>(p, s, st);
}
}  // namespace gnm
