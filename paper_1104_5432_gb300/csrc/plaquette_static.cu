// plaquette_static.cu -- the mean plaquette of one lattice with NO device
// allocation and no caller work buffer, for callers that cannot allocate
// device memory: code running inside a host framework that owns the whole
// device pool (so a cudaMalloc of its own would fail or break the
// framework's budget), or code that must not trigger the device-wide
// synchronisation a cudaMalloc/cudaFree may cause.
//
// The per-block partial sums live in a file-scope static device array of
// fixed size, so every GPU that loads the library holds these 512 KiB
// until the process exits.  All calls share that one array: two calls
// whose kernels overlap on the GPU (different streams, different host
// threads) race on it and may return wrong values; the caller must order
// them.  The array keeps the last call's contents; nothing in it has to
// start at zero because every call writes each partial it reads.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "su2.h"
#include "su2_internal.h"
#include "su2_links.cuh"
#include "su2_reduce.cuh"

namespace su2 {
namespace {

constexpr int STATIC_PARTIALS = SU2_STATIC_MAX_SITES / TPB;  // 65536 doubles = 512 KiB
constexpr int STATIC_SLOTS = STATIC_PARTIALS + 32;           // + one result slot (aligned)
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_plaq_scratch[STATIC_SLOTS];

// Device address of g_plaq_scratch for each device, looked up once per
// device with that device current.
std::mutex g_mu;
double* g_scratch_addr[MAX_DEVICES] = {};

// Variant of the stand-alone plaquette kernel: one lattice whose
// descriptor comes by value, partials into the static array.
template <typename T>
__global__ void __launch_bounds__(TPB)
plaquette_static_kernel(void* links, LatDesc D, double* __restrict__ partial)
{
    __shared__ double sred[TPB / 32];
    const uint32_t lex = blockIdx.x * TPB + threadIdx.x;
    T acc = T(0);
    if (lex < D.V) {
        const AnyLinks<T> U(links, D);
        int p;
        const EoSite s = EoSite::from_lex(D, lex, &p);
        const uint32_t eo = lex >> 1;
        const int q = p ^ 1;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const Quat<T> umu = U.load(mu, p, eo);
            const uint32_t e_pmu = s.nb(mu, +1);
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                const Quat<T> left = qmul(umu, U.load(nu, q, e_pmu));
                const Quat<T> right = qmul(U.load(nu, p, eo), U.load(mu, q, s.nb(nu, +1)));
                acc += qretr(left, qdag(right));
            }
        }
    }
    const double b = block_sum<TPB>((double)acc, sred);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

__global__ void __launch_bounds__(TPB)
plaquette_static_finalize(const double* __restrict__ partial, uint32_t nblocks, double scale,
                          double* out)
{
    __shared__ double sred[TPB / 32];
    double acc = 0.0;
    for (uint32_t b = threadIdx.x; b < nblocks; b += TPB) acc += partial[b];
    const double tot = block_sum<TPB>(acc, sred);
    if (threadIdx.x == 0) *out = tot * scale;
}

int fail_static(int code, const char* msg)
{
    char buf[256];
    snprintf(buf, sizeof buf, "su2_plaquette_static: %s", msg);
    record_error(buf);
    return code;
}

}  // namespace
}  // namespace su2

extern "C" int su2_plaquette_static(const void* links, int Ns, int Nt, int dtype, double* out,
                                    void* stream)
{
    using namespace su2;
    if (!links || !out) return fail_static(SU2_E_INVAL, "null links or output");
    if (dtype != SU2_F32 && dtype != SU2_F64 && dtype != SU2_F32_PAIRS)
        return fail_static(SU2_E_INVAL, "bad dtype");
    if (Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1))
        return fail_static(SU2_E_INVAL, "Ns and Nt must be even and >= 2");
    // bound each extent before multiplying, so no product can wrap:
    // Ns <= 256 keeps Ns^3 <= 2^24, and Ns^3 Nt then stays below 2^55
    if (Ns > 256 || Nt > SU2_STATIC_MAX_SITES)
        return fail_static(SU2_E_INVAL,
                           "lattice larger than the static scratch allows (V > 16777216)");
    const uint64_t V = (uint64_t)Ns * (uint64_t)Ns * (uint64_t)Ns * (uint64_t)Nt;
    if (V > (uint64_t)SU2_STATIC_MAX_SITES)
        return fail_static(SU2_E_INVAL,
                           "lattice larger than the static scratch allows (V > 16777216)");
    if (dtype == SU2_F32_PAIRS && Nt % 4)
        return fail_static(SU2_E_INVAL, "the site-pair layout needs Nt a multiple of 4");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(SU2_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail_static(SU2_E_INVAL, "device index too large");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_plaq_scratch);
            if (e != cudaSuccess) return fail_static(SU2_E_CUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }

    cudaPointerAttributes a;
    bool dev_out = false;
    if (cudaPointerGetAttributes(&a, out) == cudaSuccess)
        dev_out = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();

    LatDesc D;
    memset(&D, 0, sizeof D);
    D.Ns = Ns;
    D.Nt = Nt;
    D.Nh = Ns / 2;
    D.Vs = (int32_t)((uint64_t)Ns * Ns * Ns);
    D.V = (uint32_t)V;
    D.Vh = (uint32_t)(V / 2);
    D.div_nh = make_fastdiv((uint32_t)D.Nh);
    D.div_ns = make_fastdiv((uint32_t)Ns);
    D.link_off = 0;
    D.paired = dtype == SU2_F32_PAIRS ? 1 : 0;
    D.Vq = (uint32_t)(V / 4);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t nblk = (uint32_t)((V + TPB - 1) / TPB);
    void* lk = const_cast<void*>(links);
    if (dtype == SU2_F64) plaquette_static_kernel<double><<<nblk, TPB, 0, s>>>(lk, D, scratch);
    else plaquette_static_kernel<float><<<nblk, TPB, 0, s>>>(lk, D, scratch);
    double* result = scratch + STATIC_PARTIALS;
    plaquette_static_finalize<<<1, TPB, 0, s>>>(scratch, nblk, 1.0 / (6.0 * (double)V),
                                                dev_out ? out : result);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_static(SU2_E_CUDA, cudaGetErrorString(e));
    if (!dev_out) {
        e = cudaMemcpyAsync(out, result, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail_static(SU2_E_CUDA, cudaGetErrorString(e));
    }
    return SU2_OK;
}
