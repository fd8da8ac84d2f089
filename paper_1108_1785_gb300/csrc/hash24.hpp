// hash24.hpp -- hash of a /24 subnet number, shared by the host build of the /24 subnet
// table (registry.cpp) and its device probe (agg_kernel.cuh).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define GNM_HOST_DEVICE __host__ __device__
#else
#define GNM_HOST_DEVICE
#endif

namespace gnm {
GNM_HOST_DEVICE inline uint32_t hash24(uint32_t k) {
    const uint32_t h = k * 0x9E3779B1u;  // Fibonacci multiplier, then fold the high bits down
    return h ^ (h >> 15);
}
}  // namespace gnm
