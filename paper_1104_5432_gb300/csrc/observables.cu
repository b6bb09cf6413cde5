// observables.cu -- stand-alone measurements on the links:
//   mean plaquette (Sec. 2.1: "mean average plaquette"),
//   Polyakov loop L(x) = 1/2 Tr prod_t U_t(x,t) and its volume mean
//   (Sec. 2.2, Eq. 1), and the Polyakov-loop correlator
//   C(r) = <L(x) L(x + r e_i)> over x and the three spatial axes
//   (Sec. 2.2, Eq. 3: for SU(2) the traces are real, so 1/4 Tr L Tr L^+ is
//   the product of the normalised loops).
// Products are taken in the link precision, every sum in FP64 and in a
// fixed order: per-block partials, then one block per (lattice, row).
#include "su2_internal.h"
#include "su2_links.cuh"
#include "su2_reduce.cuh"

namespace su2 {

template <typename T>
__global__ void __launch_bounds__(TPB) plaquette_kernel(Ctx ctx)
{
    __shared__ double sred[TPB / 32];
    const int l = lattice_of_block(ctx.site_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t lex = (blockIdx.x - __ldg(ctx.site_start + l)) * TPB + threadIdx.x;
    T acc = T(0);
    if (lex < D.V) {
        const Links<T> U(ctx.links, D);
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
    const double b = block_sum<TPB>((double)acc, sred);
    if (threadIdx.x == 0) ctx.obs_partial[blockIdx.x] = b;
}

template <typename T>
__global__ void __launch_bounds__(TPB) polyakov_kernel(Ctx ctx)
{
    __shared__ double sred[TPB / 32];
    const int l = lattice_of_block(ctx.spat_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t sidx = (blockIdx.x - __ldg(ctx.spat_start + l)) * TPB + threadIdx.x;
    double L = 0.0;
    if (sidx < (uint32_t)D.Vs) {
        const Links<T> U(ctx.links, D);
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
        L = (double)P.a0;
        ctx.field[D.field_off + sidx] = L;
    }
    const double b = block_sum<TPB>(L, sred);
    if (threadIdx.x == 0) ctx.obs_partial[blockIdx.x] = b;
}

// rows r = 0..rmax of partials, from the Polyakov field of the last
// polyakov_kernel launch
__global__ void __launch_bounds__(TPB) correlator_kernel(Ctx ctx, int rmax)
{
    __shared__ double sred[TPB / 32];
    const int l = lattice_of_block(ctx.spat_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t sidx = (blockIdx.x - __ldg(ctx.spat_start + l)) * TPB + threadIdx.x;
    const bool act = sidx < (uint32_t)D.Vs;
    const double* F = ctx.field + D.field_off;
    uint32_t x = 0, y = 0, z = 0;
    double L0 = 0.0;
    const uint32_t Ns = (uint32_t)D.Ns;
    if (act) {
        const uint32_t r = fdiv(sidx, D.div_ns);
        x = sidx - r * Ns;
        z = fdiv(r, D.div_ns);
        y = r - z * Ns;
        L0 = F[sidx];
    }
    for (int r = 0; r <= rmax; ++r) {
        double v = 0.0;
        if (act) {
            const uint32_t xr = (x + r) % Ns, yr = (y + r) % Ns, zr = (z + r) % Ns;
            v = L0 * (F[xr + Ns * (y + Ns * z)] + F[x + Ns * (yr + Ns * z)]
                      + F[x + Ns * (y + Ns * zr)]);
        }
        const double b = block_sum<TPB>(v, sred);
        if (threadIdx.x == 0) ctx.obs_partial[(size_t)r * ctx.spat_blocks + blockIdx.x] = b;
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
                            cudaStream_t s)
{
    if (dtype == 0) polyakov_kernel<float><<<c.spat_blocks, TPB, 0, s>>>(c);
    else polyakov_kernel<double><<<c.spat_blocks, TPB, 0, s>>>(c);
    finalize_kernel<<<dim3(c.n, 1), TPB, 0, s>>>(c, c.spat_start, c.spat_blocks, 1, 1,
                                                 out_signed_dev, out_abs_dev, 0);
    return cudaGetLastError();
}

cudaError_t launch_correlator(const Ctx& c, int rmax, double* out_dev, int accumulate,
                              cudaStream_t s)
{
    correlator_kernel<<<c.spat_blocks, TPB, 0, s>>>(c, rmax);
    finalize_kernel<<<dim3(c.n, rmax + 1), TPB, 0, s>>>(c, c.spat_start, c.spat_blocks, rmax + 1,
                                                        2, out_dev, nullptr, accumulate);
    return cudaGetLastError();
}

}  // namespace su2
