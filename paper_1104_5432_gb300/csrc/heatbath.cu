// heatbath.cu -- one checkerboard phase of the SU(2) heat-bath sweep.
//
// Phase (mu, p) replaces every link U_mu(x) with parity(x) = p by a draw
// from its conditional law exp(beta k a0(U Vhat)) dU, where the staple sum
// A = k Vhat collects the six plaquettes through U_mu(x).  Links of one
// phase share no staple, so one thread per link updates them all at once.
// (The paper's benchmark, Sec. 2.1: random SU(2) start, heat-bath
// iterations, mean plaquette after each.)
//
// Per link: 18 neighbour loads (7 distinct links per update on average over
// the phase: V/2 opposite-parity U_mu plus 3V other-direction links for V/2
// updates), 12 quaternion products, the Kennedy-Pendleton draw of
// delta = 1 - a0 (one Philox block per trial), the direction (one Philox
// block), U = X A^dagger / k, renormalisation, one store.
//
// The mean plaquette after the sweep is fused in: in phase (mu, 1) with
// mu >= 1 the plane-nu part S_nu of the staple (nu < mu) closes exactly the
// plaquettes of plane (nu, mu) at the odd sites and at x - nu_hat, and every
// link of that plane is final for the sweep.  Each thread adds
// 1/2 Tr(U_new S_nu) over nu < mu; so the six planes are covered exactly once
// at no extra memory traffic.
#include "su2_internal.h"
#include "su2_links.cuh"
#include "su2_math.cuh"
#include "su2_reduce.cuh"

namespace su2 {

template <typename T> __device__ __forceinline__ T alpha_haar();
template <> __device__ __forceinline__ float alpha_haar<float>() { return 1e-12f; }
template <> __device__ __forceinline__ double alpha_haar<double>() { return 1e-12; }

// warp partial sum in the link precision (fixed butterfly order)
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int MU, bool PLAQ, bool DBG>
__global__ void __launch_bounds__(TPB, HB_MIN_BLOCKS)
hb_phase_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    __shared__ uint32_t s_trials[TPB / 32];
    __shared__ T s_plaq[TPB / 32];

    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh;
    const uint32_t blk0 = __ldg(ctx.phase_start + l);
    const uint32_t i = (blockIdx.x - blk0) * TPB + threadIdx.x;
    const bool active = i < Vh;
    const Links<T> U(ctx.links, D);
    const int q = p ^ 1;

    T plaq = T(0);
    uint32_t ntrial = 0;
    int ncap = 0;

    if (active) {
        const EoSite s(D, i, p);
        const uint32_t e_pmu = s.nb(MU, +1);

        Quat<T> A = {T(0), T(0), T(0), T(0)};
        Quat<T> Sp[MU > 0 ? MU : 1];
#pragma unroll
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == MU) continue;
            const uint32_t e_pnu = s.nb(nu, +1);
            const uint32_t e_mnu = s.nb(nu, -1);
            const uint32_t e_pmu_mnu = s.nb(MU, +1, nu, -1);
            const Quat<T> a = U.load(nu, q, e_pmu);      // U_nu(x+mu)
            const Quat<T> b = U.load(MU, q, e_pnu);      // U_mu(x+nu)
            const Quat<T> c = U.load(nu, p, i);          // U_nu(x)
            const Quat<T> d = U.load(nu, p, e_pmu_mnu);  // U_nu(x+mu-nu)
            const Quat<T> e = U.load(MU, q, e_mnu);      // U_mu(x-nu)
            const Quat<T> f = U.load(nu, q, e_mnu);      // U_nu(x-nu)
            const Quat<T> up = qmul_nd(qmul_nd(a, b), c);
            const Quat<T> lo = qmul(qmul_dd(d, e), f);
            const Quat<T> S = qadd(up, lo);
            A = qadd(A, S);
            if (PLAQ && nu < MU) Sp[nu < MU ? nu : 0] = S;
        }

        // alpha = beta k and 1/(2 alpha) from one reciprocal square root of k^2
        const T k2 = qnorm2(A);
        const T rk = Math<T>::rsqrt(k2);
        const T beta = T(D.beta);
        const T alpha = beta * k2 * rk;
        const uint64_t sw = D.sweep;
        const Stream st{(uint32_t)D.seed, (uint32_t)(D.seed >> 32), s.lex() * 4u + MU,
                        (uint32_t)sw, (uint32_t)(sw >> 32)};

        Quat<T> un;
        int32_t tr;
        if (!(alpha >= alpha_haar<T>())) {
            // alpha -> 0 limit of the conditional law (zero staple or beta = 0)
            un = haar_from<T>(st.draw(TAG_DIRECTION, 0));
            tr = 0;
        } else {
            const T inv2a = T(0.5) * rk / beta;
            T delta = T(0);
            tr = -1;
            for (int t = 0; t < KP_CAP; ++t) {
                const U4 w = st.draw(TAG_TRIAL, (uint32_t)t);
                const T r1 = u01<T>(w.x), r2 = u01<T>(w.y), r3 = u01<T>(w.z), r4 = u01<T>(w.w);
                const T lam2 = -(Math<T>::ln_u01(r1) + Math<T>::cos2pi_sq(r2) *
                                 Math<T>::ln_u01(r3)) * inv2a;
                if (r4 * r4 <= T(1) - lam2) {
                    delta = T(2) * lam2;
                    tr = t + 1;
                    break;
                }
            }
            if (tr > 0) {
                const U4 w = st.draw(TAG_DIRECTION, 0);
                const T cth = T(2) * u01<T>(w.x) - T(1);
                const T sth = Math<T>::sqrt_pos((T(1) - cth) * (T(1) + cth));
                T sph, cph;
                Math<T>::sincos2pi(u01<T>(w.y), &sph, &cph);
                const T vl = Math<T>::sqrt_pos(delta * (T(2) - delta));
                const Quat<T> X = {T(1) - delta, vl * sth * cph, vl * sth * sph, vl * cth};
                un = qnormalise(qmul_nd(X, A));
            }
        }
        if (tr >= 0) {
            U.store(MU, p, i, un);
        } else {
            ncap = 1;
            if (PLAQ) un = U.load_rw(MU, p, i);
        }
        ntrial = tr > 0 ? (uint32_t)tr : (tr < 0 ? (uint32_t)KP_CAP : 0u);
        if (DBG) dbg[s.lex()] = tr;

        if (PLAQ) {
#pragma unroll
            for (int nu = 0; nu < MU; ++nu) plaq += qretr(un, Sp[nu]);
        }
    }

    // One barrier for every block total: warp partials to shared memory,
    // cap hits counted by the barrier itself.  Trial counts are exact
    // integers (atomics); the plaquette partial is written per block and
    // summed later in a fixed order.
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wt = __reduce_add_sync(0xffffffffu, ntrial);
    T wp = T(0);
    if (PLAQ) wp = warp_sum_t(plaq);
    if (lane == 0) {
        s_trials[w] = wt;
        if (PLAQ) s_plaq[w] = wp;
    }
    const int bc = __syncthreads_count(ncap);
    if (threadIdx.x == 0) {
        unsigned long long bt = 0;
        double bp = 0.0;
#pragma unroll
        for (int k = 0; k < TPB / 32; ++k) {
            bt += s_trials[k];
            if (PLAQ) bp += (double)s_plaq[k];
        }
        if (PLAQ) ctx.plaq_partial[(size_t)(MU - 1) * ctx.phase_blocks + blockIdx.x] = bp;
        LatDesc* Dw = ctx.desc + l;
        atomicAdd(&Dw->trials, bt);
        if (blockIdx.x == blk0) atomicAdd(&Dw->updates, (unsigned long long)Vh);
        if (bc) {
            atomicAdd(&Dw->caps, (unsigned long long)bc);
            atomicOr(ctx.status, STATUS_CAP_HIT);
        }
    }
}

// Finishes a sweep: the fixed-order sum of the fused plaquette partials and
// the lattice's sweep counter.  Grid (chunks, lattices); each block sums
// SWEEP_CHUNK partials of its lattice, the last block of a lattice to finish
// (ticket counter) adds the chunk sums in chunk order.
template <bool PLAQ>
__global__ void __launch_bounds__(TPB) sweep_end_kernel(Ctx ctx)
{
    __shared__ double sred[TPB / 32];
    __shared__ int s_last;
    const int l = blockIdx.y;
    LatDesc* D = ctx.desc + l;
    if (!PLAQ) {
        if (blockIdx.x == 0 && threadIdx.x == 0) D->sweep += 1;
        return;
    }
    const uint32_t b0 = ctx.phase_start[l];
    const uint32_t nb = ctx.phase_start[l + 1] - b0;
    const uint32_t total = 3 * nb;
    const uint32_t nchunk = (total + SWEEP_CHUNK - 1) / SWEEP_CHUNK;
    if (blockIdx.x >= nchunk) return;

    const uint32_t e0 = blockIdx.x * SWEEP_CHUNK;
    const uint32_t e1 = min(e0 + (uint32_t)SWEEP_CHUNK, total);
    double acc = 0.0;
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        const uint32_t slot = (e >= nb) + (e >= 2 * nb);
        acc += ctx.plaq_partial[(size_t)slot * ctx.phase_blocks + b0 + (e - slot * nb)];
    }
    const double part = block_sum<TPB>(acc, sred);
    double* chunks = ctx.chunk_partial + (size_t)l * ctx.max_chunks;
    if (threadIdx.x == 0) {
        chunks[blockIdx.x] = part;
        __threadfence();
        const uint32_t ticket = atomicAdd(ctx.chunk_count + l, 1u);
        s_last = ticket == nchunk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double c = 0.0;
    for (uint32_t k = threadIdx.x; k < nchunk; k += TPB) c += __ldcg(chunks + k);
    const double tot = block_sum<TPB>(c, sred);
    if (threadIdx.x == 0) {
        ctx.chunk_count[l] = 0;
        const double P = tot / (6.0 * (double)D->V);
        const uint64_t k = D->sweep - D->sweep_base;
        ctx.ring[(size_t)l * PLAQ_RING + (k % PLAQ_RING)] = P;
        if (D->plaq_out) D->plaq_out[k] = P;
        D->sweep += 1;
    }
}

// Per-call parameters go in by value (no host-to-device copy); the
// plaquette index origin is the lattice's own sweep counter at call time.
__global__ void set_params_kernel(Ctx ctx, ParamChunk pc)
{
    const int j = threadIdx.x;
    if (j >= pc.count) return;
    LatDesc* D = ctx.desc + pc.first + j;
    D->beta = pc.beta[j];
    D->seed = pc.seed[j];
    D->plaq_out = pc.plaq_out[j];
    D->sweep_base = D->sweep;
}

template <typename T, int MU>
static cudaError_t launch_phase_t(const Ctx& c, int parity, bool plaq, int32_t* dbg,
                                  cudaStream_t s)
{
    const dim3 grid(c.phase_blocks), block(TPB);
    if (dbg) {
        if (plaq) hb_phase_kernel<T, MU, true, true><<<grid, block, 0, s>>>(c, parity, dbg);
        else hb_phase_kernel<T, MU, false, true><<<grid, block, 0, s>>>(c, parity, dbg);
    } else {
        if (plaq) hb_phase_kernel<T, MU, true, false><<<grid, block, 0, s>>>(c, parity, dbg);
        else hb_phase_kernel<T, MU, false, false><<<grid, block, 0, s>>>(c, parity, dbg);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_phase_mu(const Ctx& c, int mu, int parity, bool plaq, int32_t* dbg,
                                   cudaStream_t s)
{
    // the fused plaquette exists only in the odd phases with mu >= 1
    const bool pl = plaq && parity == 1 && mu >= 1;
    switch (mu) {
    case 0: return launch_phase_t<T, 0>(c, parity, false, dbg, s);
    case 1: return launch_phase_t<T, 1>(c, parity, pl, dbg, s);
    case 2: return launch_phase_t<T, 2>(c, parity, pl, dbg, s);
    default: return launch_phase_t<T, 3>(c, parity, pl, dbg, s);
    }
}

cudaError_t launch_phase(const Ctx& c, int dtype, int mu, int parity, bool plaq,
                         int32_t* dbg_trials, cudaStream_t s)
{
    if (dtype == 0) return launch_phase_mu<float>(c, mu, parity, plaq, dbg_trials, s);
    return launch_phase_mu<double>(c, mu, parity, plaq, dbg_trials, s);
}

cudaError_t launch_sweep_end(const Ctx& c, bool plaq, cudaStream_t s)
{
    if (plaq) sweep_end_kernel<true><<<dim3(c.max_chunks, c.n), TPB, 0, s>>>(c);
    else sweep_end_kernel<false><<<dim3(1, c.n), 32, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_set_params(const Ctx& c, const ParamChunk& pc, cudaStream_t s)
{
    set_params_kernel<<<1, PARAM_CHUNK, 0, s>>>(c, pc);
    return cudaGetLastError();
}

}  // namespace su2
