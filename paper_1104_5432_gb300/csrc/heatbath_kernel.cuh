// heatbath_kernel.cuh -- the checkerboard phase kernel of the SU(2) heat
// bath, templated on the link precision, the direction, the fused
// plaquette, the per-link trial output and the launch shape (threads per
// block, minimum resident blocks), so that several shapes can be compiled
// and the fastest chosen at run time (the results never depend on it).
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
// delta = 1 - a0 (one Philox block per trial; the direction comes from the
// 9 spare low bits of the four words of the first trial's block),
// U = X A^dagger / k, renormalisation, one store.
//
// The mean plaquette after the sweep is fused in: in phase (mu, 1) with
// mu >= 1 the plane-nu part S_nu of the staple (nu < mu) closes exactly the
// plaquettes of plane (nu, mu) at the odd sites and at x - nu_hat, and every
// link of that plane is final for the sweep.  Each thread adds
// 1/2 Tr(U_new S_nu) over nu < mu; so the six planes are covered exactly once
// at no extra memory traffic.
#pragma once
#include "su2_internal.h"
#include "su2_links.cuh"
#include "su2_math.cuh"
#include "su2_reduce.cuh"

namespace su2 {

template <typename T> __device__ __forceinline__ T alpha_haar();
template <> __device__ __forceinline__ float alpha_haar<float>() { return 1e-12f; }
template <> __device__ __forceinline__ double alpha_haar<double>() { return 1e-12; }

template <typename T> __device__ __forceinline__ T beta_of(const LatDesc& D);
template <> __device__ __forceinline__ float beta_of<float>(const LatDesc& D) { return D.beta_f; }
template <> __device__ __forceinline__ double beta_of<double>(const LatDesc& D) { return D.beta; }
template <typename T> __device__ __forceinline__ T creutz_of(const LatDesc& D);
template <> __device__ __forceinline__ float creutz_of<float>(const LatDesc& D) { return D.creutz_below_f; }
template <> __device__ __forceinline__ double creutz_of<double>(const LatDesc& D) { return D.creutz_below; }

// warp partial sum in the link precision (fixed butterfly order)
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int MU, bool PLAQ, bool DBG, int NT, int MINB, bool SLAB, bool HYB>
__global__ void __launch_bounds__(NT, MINB)
hb_phase_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh;
    const uint32_t blk0 = __ldg(ctx.phase_start + l);
    const uint32_t j = (blockIdx.x - blk0) * NT + threadIdx.x;  // traversal position
    const bool active = j < Vh;
    const Links<T> U(ctx.links, D);
    const int q = p ^ 1;

    T plaq = T(0);
    uint32_t ntrial = 0;
    bool ncap = false;

    if (active) {
        uint32_t i = j;  // storage index of the site
        const EoSite s = SLAB ? EoSite::from_slab(D, j, p, &i) : EoSite(D, j, p);
        int hp[4], hm[4];
        s.hops(hp, hm);
        const uint32_t e_pmu = i + hp[MU];

        Quat<T> A = {T(0), T(0), T(0), T(0)};
        Quat<T> Sp[MU > 0 ? MU : 1];
#pragma unroll
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == MU) continue;
            const uint32_t e_pnu = i + hp[nu];
            const uint32_t e_mnu = i + hm[nu];
            const uint32_t e_pmu_mnu = i + hp[MU] + hm[nu];
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
        const T beta = beta_of<T>(D);
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
            // trial 0 also carries the direction in the low 9 bits of its words
            U4 w = st.draw(TAG_TRIAL, 0u);
            const uint32_t kd1 = ((w.x & 511u) << 9) | (w.y & 511u);
            const uint32_t kd2 = ((w.z & 511u) << 9) | (w.w & 511u);
            if (HYB && alpha < creutz_of<T>(D)) {
                // Creutz's draw (small alpha, where Kennedy-Pendleton accepts
                // rarely): a0 from exp(alpha a0) by inversion, accepted with
                // sqrt(1 - a0^2); the same trial blocks, r1 = word 0, r4 = word 3
                const T q = -Math<T>::expm1(T(-2) * alpha);
                for (int t = 0; t < KP_CAP; ++t) {
                    const U4 ww = t == 0 ? w : st.draw(TAG_TRIAL, (uint32_t)t);
                    const T r1 = u01<T>(ww.x), r4 = u01<T>(ww.w);
                    const T d = -Math<T>::log1p(-r1 * q) * (T(2) * inv2a);
                    if (r4 * r4 <= d * (T(2) - d)) {
                        delta = d;
                        tr = t + 1;
                        break;
                    }
                }
            } else {
                auto kp_try = [&](const U4& ww, T* d) -> bool {
                    const T r1 = u01<T>(ww.x), r2 = u01<T>(ww.y), r3 = u01<T>(ww.z),
                            r4 = u01<T>(ww.w);
                    const T lam2 = -(Math<T>::ln_u01(r1) + Math<T>::cos2pi_sq(r2) *
                                     Math<T>::ln_u01(r3)) * inv2a;
                    *d = T(2) * lam2;
                    return r4 * r4 <= T(1) - lam2;
                };
                if (kp_try(w, &delta)) {
                    tr = 1;
                } else {
                    for (int t = 1; t < KP_CAP; ++t) {
                        if (kp_try(st.draw(TAG_TRIAL, (uint32_t)t), &delta)) {
                            tr = t + 1;
                            break;
                        }
                    }
                }
            }
            if (tr > 0) {
                const T cth = T(2) * u18<T>(kd1) - T(1);
                const T sth = Math<T>::sqrt_pos((T(1) - cth) * (T(1) + cth));
                T sph, cph;
                Math<T>::sincos2pi(u18<T>(kd2), &sph, &cph);
                const T vl = Math<T>::sqrt_pos(delta * (T(2) - delta));
                const Quat<T> X = {T(1) - delta, vl * sth * cph, vl * sth * sph, vl * cth};
                un = qnormalise(qmul_nd(X, A));
            }
        }
        if (tr >= 0) {
            U.store(MU, p, i, un);
        } else {
            ncap = true;
            if (PLAQ) un = U.load_rw(MU, p, i);
        }
        ntrial = tr > 0 ? (uint32_t)tr : (tr < 0 ? (uint32_t)KP_CAP : 0u);
        if (DBG) dbg[s.lex()] = tr;

        if (PLAQ) {
#pragma unroll
            for (int nu = 0; nu < MU; ++nu) plaq += qretr(un, Sp[nu]);
        }
    }

    // Totals without any block barrier (a warp never waits for the
    // block's slowest warp): trial counts go to spread per-lattice atomic
    // slots (exact integers), cap hits to an atomic only when present, the
    // plaquette to one partial per warp, summed later in a fixed order.
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wt = __reduce_add_sync(0xffffffffu, ntrial);
    const uint32_t capmask = __ballot_sync(0xffffffffu, ncap);
    T wp = T(0);
    if (PLAQ) wp = warp_sum_t(plaq);
    if (lane == 0) {
        const uint32_t gw = blockIdx.x * (NT / 32) + w;  // global warp index
        if (PLAQ)
            ctx.plaq_partial[(size_t)(MU - 1) * ctx.phase_blocks * (NT / 32) + gw] = (double)wp;
        atomicAdd(ctx.trial_slots + (size_t)l * TRIAL_SLOTS + (gw % TRIAL_SLOTS),
                  (unsigned long long)wt);
        LatDesc* Dw = ctx.desc + l;
        if (w == 0 && blockIdx.x == blk0) atomicAdd(&Dw->updates, (unsigned long long)Vh);
        if (capmask) {
            atomicAdd(&Dw->caps, (unsigned long long)__popc(capmask));
            atomicOr(ctx.status, STATUS_CAP_HIT);
        }
    }
}

// One launch shape (NT threads per block, at least MINB blocks per SM) of
// the phase kernel; the grid covers ctx.phase_blocks blocks of NT links.
template <typename T, int NT, int MINB, bool SLAB>
cudaError_t launch_phase_shape(const Ctx& c, int mu, int parity, bool plaq, int32_t* dbg,
                               bool hyb, cudaStream_t s)
{
    // the fused plaquette exists only in the odd phases with mu >= 1
    const bool pl = plaq && parity == 1 && mu >= 1;
    const dim3 grid(c.phase_blocks), block(NT);
#define SU2_LAUNCH_H(MUV, H)                                                                     \
    do {                                                                                         \
        if (dbg) hb_phase_kernel<T, MUV, false, true, NT, MINB, SLAB, H><<<grid, block, 0, s>>>(c, parity, dbg); \
        else if (pl) hb_phase_kernel<T, MUV, (MUV > 0), false, NT, MINB, SLAB, H><<<grid, block, 0, s>>>(c, parity, dbg); \
        else hb_phase_kernel<T, MUV, false, false, NT, MINB, SLAB, H><<<grid, block, 0, s>>>(c, parity, dbg); \
    } while (0)
#define SU2_LAUNCH(MUV)                 \
    do {                                \
        if (hyb) SU2_LAUNCH_H(MUV, true);  \
        else SU2_LAUNCH_H(MUV, false);  \
    } while (0)
    switch (mu) {
    case 0: SU2_LAUNCH(0); break;
    case 1: SU2_LAUNCH(1); break;
    case 2: SU2_LAUNCH(2); break;
    default: SU2_LAUNCH(3); break;
    }
#undef SU2_LAUNCH
#undef SU2_LAUNCH_H
    return cudaGetLastError();
}

}  // namespace su2
