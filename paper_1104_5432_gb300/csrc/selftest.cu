// selftest.cu -- exhaustive check of the FP32 transcendental forms used by
// the heat-bath draw against FP64 references, over every point of the
// uniform grid u = (k + 1/2) 2^-23, k = 0 .. 2^23 - 1.
#include "su2.h"
#include "su2_internal.h"
#include "su2_math.cuh"

namespace su2 {
namespace {

// max of non-negative doubles through their (monotone) bit patterns
__device__ __forceinline__ void atomic_max_pos(unsigned long long* dst, double v)
{
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

__global__ void math_selftest_kernel(unsigned long long* out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (1u << 23)) return;
    const float u = __fmul_rn((float)k + 0.5f, 1.1920928955078125e-7f);
    const double ud = (double)u;
    // ln u, relative error
    const double lref = log(ud);
    const double lerr = fabs((double)Math<float>::ln_u01(u) - lref) / fabs(lref);
    // cos^2(2 pi u), absolute error
    const double cref = cospi(2.0 * ud);
    const double cerr = fabs((double)Math<float>::cos2pi_sq(u) - cref * cref);
    // sin, cos (2 pi u), absolute error
    float sf, cf;
    Math<float>::sincos2pi(u, &sf, &cf);
    double sref, cref2;
    sincospi(2.0 * ud, &sref, &cref2);
    const double serr = fmax(fabs((double)sf - sref), fabs((double)cf - cref2));
    // x rsqrt(x) on the same grid, relative error
    const double qerr = fabs((double)Math<float>::sqrt_pos(u) - sqrt(ud)) / sqrt(ud);
    // block maxima via warp shuffles, then one atomic per warp
    double v[4] = {lerr, cerr, serr, qerr};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double m = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomic_max_pos(out + j, m);
    }
}

}  // namespace
}  // namespace su2

extern "C" int su2_selftest_math(void* out, void* stream)
{
    if (!out) return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out, 0, 4 * sizeof(double), s) != cudaSuccess) return SU2_E_CUDA;
    su2::math_selftest_kernel<<<(1u << 23) / 256, 256, 0, s>>>(
        static_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? SU2_OK : SU2_E_CUDA;
}
