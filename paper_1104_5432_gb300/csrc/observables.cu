// observables.cu -- stand-alone measurements on the links:
//   mean plaquette (Sec. 2.1: "mean average plaquette"),
//   Polyakov loop L(x) = 1/2 Tr prod_t U_t(x,t) and its volume mean
//   (Sec. 2.2, Eq. 1), and the Polyakov-loop correlator
//   C(r) = <L(x) L(x + r e_i)> over x and the three spatial axes
//   (Sec. 2.2, Eq. 3: for SU(2) the traces are real, so 1/4 Tr L Tr L^+ is
//   the product of the normalised loops).
// Products and warp partial sums are taken in the link precision; block,
// lattice and over-sweep sums in FP64, each in a fixed order (per-block
// partials, then one block per (lattice, row)).
#include "su2_internal.h"
#include "su2_links.cuh"
#include "su2_reduce.cuh"

namespace su2 {

template <typename T>
__device__ __forceinline__ T warp_total(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block total of one value per thread: warp sums in T, block sum in FP64
// (valid in thread 0)
template <typename T>
__device__ __forceinline__ double block_total(T v, T* s_warp)
{
    v = warp_total(v);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < TPB / 32; ++w) s += (double)s_warp[w];
    }
    return s;
}

template <typename T>
__global__ void __launch_bounds__(TPB) plaquette_kernel(Ctx ctx)
{
    __shared__ T s_warp[TPB / 32];
    const int l = lattice_of_block(ctx.site_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t lex = (blockIdx.x - first_block(ctx.site_start, l)) * TPB + threadIdx.x;
    T acc = T(0);
    if (lex < D.V) {
        const AnyLinks<T> U(ctx.links, D, ctx.status);
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
                // 1/2 Tr U_mu(x) U_nu(x+mu) [U_nu(x) U_mu(x+nu)]^+
                const Quat<T> left = qmul(umu, U.load(nu, q, e_pmu));
                const Quat<T> right = qmul(U.load(nu, p, eo), U.load(mu, q, s.nb(nu, +1)));
                acc += qretr(left, qdag(right));
            }
        }
    }
    const double b = block_total(acc, s_warp);
    if (threadIdx.x == 0) ctx.obs_partial[blockIdx.x] = b;
}

// L(x) for every spatial site into the field (link precision) and the
// per-block partial sums of L
template <typename T>
__global__ void __launch_bounds__(TPB) polyakov_kernel(Ctx ctx)
{
    __shared__ T s_warp[TPB / 32];
    const int l = lattice_of_block(ctx.spat_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t sidx = (blockIdx.x - first_block(ctx.spat_start, l)) * TPB + threadIdx.x;
    T L = T(0);
    if (sidx < (uint32_t)D.Vs) {
        const AnyLinks<T> U(ctx.links, D, ctx.status);
        const uint32_t r = fdiv(sidx, D.div_ns);
        const uint32_t x = sidx - r * (uint32_t)D.Ns;
        const uint32_t z = fdiv(r, D.div_ns);
        const uint32_t y = r - z * (uint32_t)D.Ns;
        Quat<T> P = {T(1), T(0), T(0), T(0)};
        for (int t = 0; t < D.Nt; ++t) {
            const uint32_t lex = sidx + (uint32_t)D.Vs * (uint32_t)t;
            const int p = (int)((x + y + z + (uint32_t)t) & 1u);
            P = qmul(P, U.load(3, p, lex >> 1));
        }
        L = P.a0;
        reinterpret_cast<T*>(ctx.field)[D.field_off + sidx] = L;
    }
    const double b = block_total(L, s_warp);
    if (threadIdx.x == 0) ctx.obs_partial[blockIdx.x] = b;
}

// rows r = 0..rmax of partials, from the Polyakov field of the last
// polyakov_kernel launch; one barrier for all rows
template <typename T>
__global__ void __launch_bounds__(TPB) correlator_kernel(Ctx ctx, int rmax)
{
    __shared__ T s_rows[MAX_RMAX + 1][TPB / 32];
    const int l = lattice_of_block(ctx.spat_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t sidx = (blockIdx.x - first_block(ctx.spat_start, l)) * TPB + threadIdx.x;
    const bool act = sidx < (uint32_t)D.Vs;
    const T* F = reinterpret_cast<const T*>(ctx.field) + D.field_off;
    uint32_t x = 0, y = 0, z = 0;
    T L0 = T(0);
    const uint32_t Ns = (uint32_t)D.Ns;
    if (act) {
        const uint32_t r = fdiv(sidx, D.div_ns);
        x = sidx - r * Ns;
        z = fdiv(r, D.div_ns);
        y = r - z * Ns;
        L0 = F[sidx];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t xr = x, yr = y, zr = z;
    for (int r = 0; r <= rmax; ++r) {
        T v = T(0);
        if (act) {
            v = L0 * (F[xr + Ns * (y + Ns * z)] + F[x + Ns * (yr + Ns * z)]
                      + F[x + Ns * (y + Ns * zr)]);
        }
        v = warp_total(v);
        if (lane == 0) s_rows[r][w] = v;
        xr = xr + 1 == Ns ? 0 : xr + 1;
        yr = yr + 1 == Ns ? 0 : yr + 1;
        zr = zr + 1 == Ns ? 0 : zr + 1;
    }
    __syncthreads();
    if ((int)threadIdx.x <= rmax) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < TPB / 32; ++k) s += (double)s_rows[threadIdx.x][k];
        ctx.obs_partial[(size_t)threadIdx.x * ctx.spat_blocks + blockIdx.x] = s;
    }
}

// out[l*rows + row] (=|+=) scale_l * sum of the lattice's partials in row
// `row`; mode 0: scale 1/(6V) (plaquette), 1: 1/Vs (Polyakov), 2: 1/(3Vs)
// (correlator).  abs_out (nullable, mode 1) gets |mean|.
__global__ void __launch_bounds__(TPB)
finalize_kernel(Ctx ctx, const uint32_t* __restrict__ start, uint32_t stride, int rows, int mode,
                double* out, double* abs_out, int accumulate)
{
    __shared__ double sred[TPB / 32];
    const int l = blockIdx.x, row = blockIdx.y;
    const LatDesc& D = ctx.desc[l];
    const uint32_t b0 = start[l], b1 = start[l + 1];
    double acc = 0.0;
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += TPB)
        acc += ctx.obs_partial[(size_t)row * stride + b];
    const double tot = block_sum<TPB>(acc, sred);
    if (threadIdx.x == 0) {
        const double scale = mode == 0 ? 1.0 / (6.0 * (double)D.V)
                           : mode == 1 ? 1.0 / (double)D.Vs
                                       : 1.0 / (3.0 * (double)D.Vs);
        const double v = tot * scale;
        double* o = out + (size_t)l * rows + row;
        *o = accumulate ? *o + v : v;
        if (abs_out) {
            double* a = abs_out + l;
            *a = accumulate ? *a + fabs(v) : fabs(v);
        }
    }
}

cudaError_t launch_plaquette(const Ctx& c, int dtype, double* out_dev, cudaStream_t s)
{
    if (dtype == 0) plaquette_kernel<float><<<c.site_blocks, TPB, 0, s>>>(c);
    else plaquette_kernel<double><<<c.site_blocks, TPB, 0, s>>>(c);
    finalize_kernel<<<dim3(c.n, 1), TPB, 0, s>>>(c, c.site_start, c.site_blocks, 1, 0, out_dev,
                                                 nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_polyakov(const Ctx& c, int dtype, double* out_signed_dev, double* out_abs_dev,
                            int accumulate, cudaStream_t s)
{
    if (dtype == 0) polyakov_kernel<float><<<c.spat_blocks, TPB, 0, s>>>(c);
    else polyakov_kernel<double><<<c.spat_blocks, TPB, 0, s>>>(c);
    finalize_kernel<<<dim3(c.n, 1), TPB, 0, s>>>(c, c.spat_start, c.spat_blocks, 1, 1,
                                                 out_signed_dev, out_abs_dev, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_correlator(const Ctx& c, int dtype, int rmax, double* out_dev, int accumulate,
                              cudaStream_t s)
{
    if (dtype == 0) correlator_kernel<float><<<c.spat_blocks, TPB, 0, s>>>(c, rmax);
    else correlator_kernel<double><<<c.spat_blocks, TPB, 0, s>>>(c, rmax);
    finalize_kernel<<<dim3(c.n, rmax + 1), TPB, 0, s>>>(c, c.spat_start, c.spat_blocks, rmax + 1,
                                                        2, out_dev, nullptr, accumulate);
    return cudaGetLastError();
}

}  // namespace su2
