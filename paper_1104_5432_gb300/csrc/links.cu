// links.cu -- start configurations, conversion between the device layout
// and the canonical host layout double[V][4][4] ([lex][mu][a0..a3]), and
// the random gauge transformation used to check gauge invariance.
//
// Hot start: "random SU(2) matrix initialization" (Sec. 2.1), read as
// Haar-distributed links: four normals from one Philox block (tag 2,
// counter (lex*4+mu, 0, 2<<24, 0)), normalised onto S^3.
#include <type_traits>

#include "su2_internal.h"
#include "su2_links.cuh"

namespace su2 {

template <typename T>
__device__ __forceinline__ Quat<T> start_link(int hot, uint64_t seed, uint32_t lex, int mu)
{
    if (!hot) return {T(1), T(0), T(0), T(0)};
    const Stream st{(uint32_t)seed, (uint32_t)(seed >> 32), lex * 4u + (uint32_t)mu, 0u, 0u};
    return haar_from<T>(st.draw(TAG_HOT, 0));
}

// one lattice, one thread per site (per site pair on a paired FP32
// lattice: lex and lex + V/2, written as whole records); also clears the
// lattice's counters
template <typename T>
__global__ void __launch_bounds__(TPB) init_kernel(Ctx ctx, int l, int hot, uint64_t seed)
{
    LatDesc* Dw = ctx.desc + l;
    const LatDesc& D = *Dw;
    const uint32_t lex = blockIdx.x * TPB + threadIdx.x;
    if (lex == 0) {
        Dw->sweep = 0;
        Dw->trials = Dw->updates = Dw->caps = 0;
    }
    if (lex < TRIAL_SLOTS) ctx.trial_slots[(size_t)l * TRIAL_SLOTS + lex] = 0;
    int p;
    if constexpr (std::is_same<T, float>::value) {
        if (D.paired) {
            if (lex >= D.V / 2) return;
            const PairLinks U(ctx.links, D, ctx.status);
            EoSite::from_lex(D, lex, &p);  // lex + V/2 has the same parity (Nt/2 even)
            for (int mu = 0; mu < 4; ++mu) {
                const Quat<float> a = start_link<float>(hot, seed, lex, mu);
                const Quat<float> b = start_link<float>(hot, seed, lex + D.V / 2, mu);
                U.store2(mu, p, lex >> 1,
                         {make_float2(a.a0, b.a0), make_float2(a.a1, b.a1),
                          make_float2(a.a2, b.a2), make_float2(a.a3, b.a3)});
            }
            return;
        }
    }
    if (lex >= D.V) return;
    const Links<T> U(ctx.links, D, ctx.status);
    EoSite::from_lex(D, lex, &p);
    for (int mu = 0; mu < 4; ++mu) U.store(mu, p, lex >> 1, start_link<T>(hot, seed, lex, mu));
}

// Canonical <-> device layout, 64 sites per block: the block's part of the
// canonical array (16 values of type C per site: 8 KB for double, 4 KB for
// float) moves as 16-byte vectors with consecutive threads on consecutive
// addresses (so the source or target may as well be page-locked host
// memory read or written directly over the host link), and is reordered in
// shared memory; thread (site k, direction mu) then reads or writes one
// link.
constexpr int CANON_SITES = TPB / 4;

template <typename T, typename C>
__global__ void __launch_bounds__(TPB)
to_canonical_kernel(Ctx ctx, int l, uint32_t lex0, uint32_t nsite, C* __restrict__ dst)
{
    constexpr int CH = (int)sizeof(C);  // 16-byte chunks per site
    __shared__ uint4 sh[CANON_SITES * CH];
    C* shc = reinterpret_cast<C*>(sh);
    const LatDesc& D = ctx.desc[l];
    const uint32_t s0 = blockIdx.x * CANON_SITES;
    const uint32_t cnt = min((uint32_t)CANON_SITES, nsite - s0);
    const uint32_t k = threadIdx.x >> 2;
    const int mu = threadIdx.x & 3;
    if (k < cnt) {
        const uint32_t lex = lex0 + s0 + k;
        const AnyLinks<T> U(ctx.links, D, ctx.status);
        int p;
        EoSite::from_lex(D, lex, &p);
        const Quat<T> a = U.load_rw(mu, p, lex >> 1);
        C* o = shc + k * 16 + mu * 4;
        o[0] = (C)a.a0;
        o[1] = (C)a.a1;
        o[2] = (C)a.a2;
        o[3] = (C)a.a3;
    }
    __syncthreads();
    uint4* out = reinterpret_cast<uint4*>(dst + (size_t)s0 * 16);
    for (uint32_t q = threadIdx.x; q < cnt * CH; q += TPB) out[q] = sh[q];
}

template <typename T, typename C>
__global__ void __launch_bounds__(TPB)
from_canonical_kernel(Ctx ctx, int l, uint32_t lex0, uint32_t nsite, const C* __restrict__ src)
{
    constexpr int CH = (int)sizeof(C);
    __shared__ uint4 sh[CANON_SITES * CH];
    const C* shc = reinterpret_cast<const C*>(sh);
    const LatDesc& D = ctx.desc[l];
    const uint32_t s0 = blockIdx.x * CANON_SITES;
    const uint32_t cnt = min((uint32_t)CANON_SITES, nsite - s0);
    const uint4* in = reinterpret_cast<const uint4*>(src + (size_t)s0 * 16);
    for (uint32_t q = threadIdx.x; q < cnt * CH; q += TPB) sh[q] = in[q];
    __syncthreads();
    const uint32_t k = threadIdx.x >> 2;
    const int mu = threadIdx.x & 3;
    if (k >= cnt) return;
    const uint32_t lex = lex0 + s0 + k;
    const AnyLinks<T> U(ctx.links, D, ctx.status);
    int p;
    EoSite::from_lex(D, lex, &p);
    const C* v = shc + k * 16 + mu * 4;
    U.store(mu, p, lex >> 1, Quat<T>{(T)v[0], (T)v[1], (T)v[2], (T)v[3]});
}

// The same conversions for a whole lattice stored as FP32 site pairs: block
// b takes the 64 sites from lex = 64 b and the 64 from lex = 64 b + V/2
// (two contiguous pieces of the canonical array, still moved as 16-byte
// vectors), so that each thread reads or writes whole 32-byte records.
template <typename C>
__global__ void __launch_bounds__(TPB)
to_canonical_pairs_kernel(Ctx ctx, int l, C* __restrict__ dst)
{
    constexpr int CH = (int)sizeof(C);
    __shared__ uint4 sh[2][CANON_SITES * CH];
    const LatDesc& D = ctx.desc[l];
    const uint32_t half = D.V / 2;
    const uint32_t s0 = blockIdx.x * CANON_SITES;
    const uint32_t cnt = min((uint32_t)CANON_SITES, half - s0);
    const uint32_t k = threadIdx.x >> 2;
    const int mu = threadIdx.x & 3;
    if (k < cnt) {
        const uint32_t lex = s0 + k;
        const PairLinks U(ctx.links, D, ctx.status);
        int p;
        EoSite::from_lex(D, lex, &p);
        const size_t i = U.ridx(mu, p, lex >> 1);
        const float4 lo = U.base[i], hi = U.base[i + 1];
        C* o0 = reinterpret_cast<C*>(sh[0]) + k * 16 + mu * 4;
        C* o1 = reinterpret_cast<C*>(sh[1]) + k * 16 + mu * 4;
        o0[0] = (C)lo.x; o0[1] = (C)lo.z; o0[2] = (C)hi.x; o0[3] = (C)hi.z;
        o1[0] = (C)lo.y; o1[1] = (C)lo.w; o1[2] = (C)hi.y; o1[3] = (C)hi.w;
    }
    __syncthreads();
    uint4* out0 = reinterpret_cast<uint4*>(dst + (size_t)s0 * 16);
    uint4* out1 = reinterpret_cast<uint4*>(dst + ((size_t)s0 + half) * 16);
    for (uint32_t q = threadIdx.x; q < cnt * CH; q += TPB) {
        out0[q] = sh[0][q];
        out1[q] = sh[1][q];
    }
}

template <typename C>
__global__ void __launch_bounds__(TPB)
from_canonical_pairs_kernel(Ctx ctx, int l, const C* __restrict__ src)
{
    constexpr int CH = (int)sizeof(C);
    __shared__ uint4 sh[2][CANON_SITES * CH];
    const LatDesc& D = ctx.desc[l];
    const uint32_t half = D.V / 2;
    const uint32_t s0 = blockIdx.x * CANON_SITES;
    const uint32_t cnt = min((uint32_t)CANON_SITES, half - s0);
    const uint4* in0 = reinterpret_cast<const uint4*>(src + (size_t)s0 * 16);
    const uint4* in1 = reinterpret_cast<const uint4*>(src + ((size_t)s0 + half) * 16);
    for (uint32_t q = threadIdx.x; q < cnt * CH; q += TPB) {
        sh[0][q] = in0[q];
        sh[1][q] = in1[q];
    }
    __syncthreads();
    const uint32_t k = threadIdx.x >> 2;
    const int mu = threadIdx.x & 3;
    if (k >= cnt) return;
    const uint32_t lex = s0 + k;
    const PairLinks U(ctx.links, D, ctx.status);
    int p;
    EoSite::from_lex(D, lex, &p);
    const C* v0 = reinterpret_cast<const C*>(sh[0]) + k * 16 + mu * 4;
    const C* v1 = reinterpret_cast<const C*>(sh[1]) + k * 16 + mu * 4;
    U.store2(mu, p, lex >> 1,
             {make_float2((float)v0[0], (float)v1[0]), make_float2((float)v0[1], (float)v1[1]),
              make_float2((float)v0[2], (float)v1[2]), make_float2((float)v0[3], (float)v1[3])});
}

// U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger, g Haar from Philox tag 3 with
// counter (lex*4, 0, 3<<24, 0).  In place: each thread reads and writes
// only the four links leaving its site; g is recomputed where needed.
template <typename T>
__global__ void __launch_bounds__(TPB) gauge_kernel(Ctx ctx, int l, uint64_t seed)
{
    const LatDesc& D = ctx.desc[l];
    const uint32_t lex = blockIdx.x * TPB + threadIdx.x;
    if (lex >= D.V) return;
    const AnyLinks<T> U(ctx.links, D, ctx.status);
    int p;
    const EoSite s = EoSite::from_lex(D, lex, &p);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const Quat<T> g = haar_from<T>(Stream{k0, k1, lex * 4u, 0u, 0u}.draw(TAG_GAUGE, 0));
    for (int mu = 0; mu < 4; ++mu) {
        // lex of x + mu
        int c[4] = {s.c[0], s.c[1], s.c[2], s.c[3]};
        c[mu] = (c[mu] + 1) % (mu == 3 ? D.Nt : D.Ns);
        const uint32_t lex_n =
            (uint32_t)c[0] + (uint32_t)D.Ns * ((uint32_t)c[1] + (uint32_t)D.Ns *
                                               ((uint32_t)c[2] + (uint32_t)D.Ns * (uint32_t)c[3]));
        const Quat<T> gn = haar_from<T>(Stream{k0, k1, lex_n * 4u, 0u, 0u}.draw(TAG_GAUGE, 0));
        const Quat<T> u = U.load_rw(mu, p, lex >> 1);
        U.store(mu, p, lex >> 1, qmul_nd(qmul(g, u), gn));
    }
}

static unsigned nblk(uint32_t n) { return (n + TPB - 1) / TPB; }
static unsigned nblk_canon(uint32_t n) { return (n + CANON_SITES - 1) / CANON_SITES; }

cudaError_t launch_init(const Ctx& c, int dtype, int l, uint32_t V, int hot, uint64_t seed,
                        cudaStream_t s)
{
    if (dtype == 0) init_kernel<float><<<nblk(V), TPB, 0, s>>>(c, l, hot, seed);
    else init_kernel<double><<<nblk(V), TPB, 0, s>>>(c, l, hot, seed);
    return cudaGetLastError();
}

// buf: device memory, or the device address of page-locked host memory;
// 16-byte aligned; canonical values in double (cdtype 1) or float (0)
cudaError_t launch_links_to_canonical(const Ctx& c, int dtype, int l, uint32_t lex0,
                                      uint32_t nsite, void* buf, int cdtype, cudaStream_t s,
                                      bool pairs_whole)
{
    if (nsite == 0) return cudaSuccess;
    if (pairs_whole) {  // the whole lattice, stored as FP32 site pairs
        const unsigned gp = nblk_canon(nsite / 2);
        if (cdtype == 1) to_canonical_pairs_kernel<double><<<gp, TPB, 0, s>>>(c, l, (double*)buf);
        else to_canonical_pairs_kernel<float><<<gp, TPB, 0, s>>>(c, l, (float*)buf);
        return cudaGetLastError();
    }
    const unsigned g = nblk_canon(nsite);
    if (dtype == 0 && cdtype == 1)
        to_canonical_kernel<float, double><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (double*)buf);
    else if (dtype == 0)
        to_canonical_kernel<float, float><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (float*)buf);
    else if (cdtype == 1)
        to_canonical_kernel<double, double><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (double*)buf);
    else
        to_canonical_kernel<double, float><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (float*)buf);
    return cudaGetLastError();
}

cudaError_t launch_links_from_canonical(const Ctx& c, int dtype, int l, uint32_t lex0,
                                        uint32_t nsite, const void* buf, int cdtype,
                                        cudaStream_t s, bool pairs_whole)
{
    if (nsite == 0) return cudaSuccess;
    if (pairs_whole) {
        const unsigned gp = nblk_canon(nsite / 2);
        if (cdtype == 1)
            from_canonical_pairs_kernel<double><<<gp, TPB, 0, s>>>(c, l, (const double*)buf);
        else
            from_canonical_pairs_kernel<float><<<gp, TPB, 0, s>>>(c, l, (const float*)buf);
        return cudaGetLastError();
    }
    const unsigned g = nblk_canon(nsite);
    if (dtype == 0 && cdtype == 1)
        from_canonical_kernel<float, double><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (const double*)buf);
    else if (dtype == 0)
        from_canonical_kernel<float, float><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (const float*)buf);
    else if (cdtype == 1)
        from_canonical_kernel<double, double><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (const double*)buf);
    else
        from_canonical_kernel<double, float><<<g, TPB, 0, s>>>(c, l, lex0, nsite, (const float*)buf);
    return cudaGetLastError();
}

cudaError_t launch_gauge(const Ctx& c, int dtype, int l, uint32_t V, uint64_t seed, cudaStream_t s)
{
    if (dtype == 0) gauge_kernel<float><<<nblk(V), TPB, 0, s>>>(c, l, seed);
    else gauge_kernel<double><<<nblk(V), TPB, 0, s>>>(c, l, seed);
    return cudaGetLastError();
}

}  // namespace su2
