// su2_reduce.cuh -- deterministic warp and block reductions.  Every sum
// is taken in a fixed order (butterfly inside a warp, then warps in index
// order), so a result depends only on the launch shape, never on timing.
#pragma once
#include <cstdint>

namespace su2 {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
    return __reduce_add_sync(0xffffffffu, v);
}

// Sum of one double per thread; the result is valid in thread 0.
// `scratch` holds at least blockDim.x / 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) scratch[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += scratch[i];
    }
    __syncthreads();
    return s;
}

template <int NT>
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* scratch)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) scratch[w] = v;
    __syncthreads();
    uint32_t s = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += scratch[i];
    }
    __syncthreads();
    return s;
}

}  // namespace su2
