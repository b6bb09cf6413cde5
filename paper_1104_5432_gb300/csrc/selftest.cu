// selftest.cu -- exhaustive check of the FP32 transcendental forms used by
// the heat-bath draw against FP64 references, over every point of the
// uniform grid u = (k + 1/2) 2^-23, k = 0 .. 2^23 - 1; and the FMA-rate
// and FP64 math-function probes that give the arithmetic rooflines their
// measured denominators (declared in su2_testing.h).
#include "su2_testing.h"
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

__device__ double fma_rate_sink;

// the FP64 path's logarithm table for the self-test and the probe (the
// heat-bath kernels read the copy in the handle's work memory)
__device__ double2 g_fp64_tab[FP64_TABLE_ENTRIES];

int upload_fp64_table()
{
    double2 tab[FP64_TABLE_ENTRIES];
    fill_fp64_table(tab);
    return cudaMemcpyToSymbol(g_fp64_tab, tab, sizeof tab) == cudaSuccess ? SU2_OK : SU2_E_CUDA;
}

// sincospi_tab against CUDA's sincospi: out[0] the cosine's largest
// absolute error on the trials' grid y = (2k + 1) 2^-23 (k < 2^23), out[1]
// the sine's and cosine's on the direction's grid y = (2k + 1) 2^-18
// (k < 2^18)
__global__ void trig_selftest_kernel(unsigned long long* out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (1u << 23)) return;
    double sn, cs, sref, cref;
    sincospi_tab(2u * k + 1u, 23, g_fp64_tab, &sn, &cs);
    sincospi(ldexp((double)(2u * k + 1u), -23), &sref, &cref);
    double v[2] = {fabs(cs - cref), 0.0};
    if (k < (1u << 18)) {
        sincospi_tab(2u * k + 1u, 18, g_fp64_tab, &sn, &cs);
        sincospi(ldexp((double)(2u * k + 1u), -18), &sref, &cref);
        v[1] = fmax(fabs(sn - sref), fabs(cs - cref));
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        double m = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomic_max_pos(out + j, m);
    }
}

// ln_u01_tab against CUDA's log on every grid point u = (2k + 1) 2^-24:
// out[0] max absolute error, out[1] max error in units of the last place of
// the reference
__global__ void ln_selftest_kernel(unsigned long long* out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (1u << 23)) return;
    const uint32_t w = k << 9;
    const double ref = log(u01d(w));
    const double err = fabs(ln_u01_tab(w, g_fp64_tab) - ref);
    const int ex = (int)((__double_as_longlong(ref) >> 52) & 0x7FF) - 1023;
    const double ulps = err / ldexp(1.0, ex - 52);
    double v[2] = {err, ulps};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        double m = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomic_max_pos(out + j, m);
    }
}

// 8 independent FMA chains per thread: the pipe never waits on a result
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == T(-1)) fma_rate_sink = (double)s;  // never true here; keeps the chains live
}

// 8 independent chains of one FP64 math function per thread, each call fed
// by the previous result so that none can be hoisted or removed
template <int FN>
__global__ void __launch_bounds__(256) special_rate_kernel(int iters)
{
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.25 + 1e-3 * (double)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (FN == SU2_PROBE_LOG) x[j] = log(x[j] + 2.0);
            else if (FN == SU2_PROBE_LN_TABLE)
                x[j] = ln_u01_tab((uint32_t)__double_as_longlong(x[j]), g_fp64_tab);
            else if (FN == SU2_PROBE_COS_TABLE || FN == SU2_PROBE_SINCOS_TABLE) {
                // an odd numerator below 2^24 from the previous result's bits
                const uint32_t num = ((uint32_t)__double_as_longlong(x[j]) & 0xFFFFFEu) | 1u;
                double sn, cs;
                sincospi_tab(num, 23, g_fp64_tab, &sn, &cs);
                x[j] = FN == SU2_PROBE_COS_TABLE ? cs : sn + cs;
            }
            else if (FN == SU2_PROBE_COSPI) x[j] = cospi(x[j]);
            else if (FN == SU2_PROBE_SINCOSPI) {
                double sn, cs;
                sincospi(x[j], &sn, &cs);
                x[j] = sn + cs;
            } else if (FN == SU2_PROBE_SQRT) x[j] = sqrt(x[j]);
            else x[j] = rsqrt(x[j]);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0) fma_rate_sink = s;  // never true here; keeps the chains live
}

// launch `blocks` blocks twice on s, time the second launch
template <typename F>
int time_probe(F launch, cudaStream_t s, float* ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return SU2_E_CUDA;
    }
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
    }
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || *ms <= 0.0f) return SU2_E_CUDA;
    return SU2_OK;
}

int probe_blocks(unsigned* blocks)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SU2_E_CUDA;
    *blocks = (unsigned)sms * 8u;
    return SU2_OK;
}

}  // namespace
}  // namespace su2

extern "C" int su2_probe_special_rate(int fn, int iters, double* calls_per_s, void* stream)
{
    if (!calls_per_s || iters <= 0 || fn < SU2_PROBE_LOG || fn > SU2_PROBE_SINCOS_TABLE)
        return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned blocks = 0;
    if (int rc = su2::probe_blocks(&blocks)) return rc;
    if (fn >= SU2_PROBE_LN_TABLE)
        if (int rc = su2::upload_fp64_table()) return rc;
    float ms = 0.0f;
    auto launch = [&] {
        switch (fn) {
        case SU2_PROBE_LOG: su2::special_rate_kernel<SU2_PROBE_LOG><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_COSPI: su2::special_rate_kernel<SU2_PROBE_COSPI><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_SINCOSPI: su2::special_rate_kernel<SU2_PROBE_SINCOSPI><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_SQRT: su2::special_rate_kernel<SU2_PROBE_SQRT><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_LN_TABLE: su2::special_rate_kernel<SU2_PROBE_LN_TABLE><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_COS_TABLE: su2::special_rate_kernel<SU2_PROBE_COS_TABLE><<<blocks, 256, 0, s>>>(iters); break;
        case SU2_PROBE_SINCOS_TABLE: su2::special_rate_kernel<SU2_PROBE_SINCOS_TABLE><<<blocks, 256, 0, s>>>(iters); break;
        default: su2::special_rate_kernel<SU2_PROBE_RSQRT><<<blocks, 256, 0, s>>>(iters); break;
        }
    };
    if (int rc = su2::time_probe(launch, s, &ms)) return rc;
    *calls_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
    return SU2_OK;
}

extern "C" int su2_probe_fma_rate(int dtype, int iters, double* fma_per_s, void* stream)
{
    if (!fma_per_s || iters <= 0 || (dtype != SU2_F32 && dtype != SU2_F64)) return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned blocks = 0;
    if (int rc = su2::probe_blocks(&blocks)) return rc;
    float ms = 0.0f;
    auto launch = [&] {
        if (dtype == SU2_F32)
            su2::fma_rate_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.999f, 1e-4f);
        else
            su2::fma_rate_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.999, 1e-4);
    };
    if (int rc = su2::time_probe(launch, s, &ms)) return rc;
    *fma_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
    return SU2_OK;
}

extern "C" int su2_selftest_math(void* out, void* stream)
{
    if (!out) return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out, 0, 4 * sizeof(double), s) != cudaSuccess) return SU2_E_CUDA;
    su2::math_selftest_kernel<<<(1u << 23) / 256, 256, 0, s>>>(
        static_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? SU2_OK : SU2_E_CUDA;
}

extern "C" int su2_selftest_ln(void* out, void* stream)
{
    if (!out) return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = su2::upload_fp64_table()) return rc;
    if (cudaMemsetAsync(out, 0, 2 * sizeof(double), s) != cudaSuccess) return SU2_E_CUDA;
    su2::ln_selftest_kernel<<<(1u << 23) / 256, 256, 0, s>>>(
        static_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? SU2_OK : SU2_E_CUDA;
}

extern "C" int su2_selftest_trig(void* out, void* stream)
{
    if (!out) return SU2_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = su2::upload_fp64_table()) return rc;
    if (cudaMemsetAsync(out, 0, 2 * sizeof(double), s) != cudaSuccess) return SU2_E_CUDA;
    su2::trig_selftest_kernel<<<(1u << 23) / 256, 256, 0, s>>>(
        static_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? SU2_OK : SU2_E_CUDA;
}
