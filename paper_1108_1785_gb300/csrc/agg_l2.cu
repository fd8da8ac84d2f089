// agg_l2.cu -- aggregation kernel variants for one prefix-match mode (see agg_kernel.cuh).
#include "agg_kernel.cuh"

namespace gnm {
cudaError_t launch_aggregate_l2(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    return dev::launch_lookup_mode<kLookupL2>(p, s, st);
}
}  // namespace gnm
