// heatbath_kernel.cuh -- the checkerboard phase kernels of the SU(2) heat
// bath, templated on the link precision, the direction, the fused
// plaquette, the per-link trial output and the launch shape (threads per
// block, minimum resident blocks, links per thread), so that several
// shapes can be compiled and the fastest chosen at run time (the results
// never depend on it).
//
// Phase (mu, p) replaces every link U_mu(x) with parity(x) = p by a draw
// from its conditional law exp(beta k a0(U Vhat)) dU, where the staple sum
// A = k Vhat collects the six plaquettes through U_mu(x).  Links of one
// phase share no staple, so all of them are updated at once.
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
// link of that plane is final for the sweep.  Each link adds
// 1/2 Tr(U_new P) with P = sum over nu < mu of S_nu (the trace is linear),
// so the six planes are covered exactly once at no extra memory traffic.
#pragma once
#include <type_traits>

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
// 1/(2 alpha) from rk = 1/k times the lattice's precomputed 1/(2 beta) (no
// division per update; 1/(2 beta) is rounded once per call in each precision)
template <typename T>
__device__ __forceinline__ T inv_two_alpha(const LatDesc& D, T rk, T beta);
template <>
__device__ __forceinline__ float inv_two_alpha<float>(const LatDesc& D, float rk, float)
{
    return mul_(rk, D.half_inv_beta_f);
}
template <>
__device__ __forceinline__ double inv_two_alpha<double>(const LatDesc& D, double rk, double)
{
    return mul_(rk, D.half_inv_beta);
}
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

// ---------------------------------------------------------------------------
// pieces shared by the two phase kernels
// ---------------------------------------------------------------------------

// Staple sum A = sum over nu != mu of the upper and lower staples of
// U_mu(x), and (PLAQ) its part P over nu < mu, which closes the plaquettes
// of the planes (nu, mu).  P is A after its first mu terms, so it costs no
// extra additions.
//
// The order of the additions is fixed per precision, and every kernel of a
// precision keeps it, so all launch shapes give the same bits.  FP32 folds
// the sums into the products' last multiply-adds (A = A + up + lo, ν by ν).
// FP64 sums a tree: s_k = up_k + lo_k for the k-th ν != mu, then
// A = (s_0 + s_1) + s_2 (P = the prefix over ν < mu), the order in which
// the cooperative kernel's lanes, which compute the six terms in parallel,
// can reproduce it.
template <int MU>
__device__ __forceinline__ constexpr int nu_of(int k) { return k + (k >= MU ? 1 : 0); }

// the upper (a b^dagger c^dagger) or lower ((e d)^dagger f) staple term of
// U_mu(x) in the plane (nu, mu).  Both are formed as x y^dagger z^dagger:
// the lower one is d^dagger e^dagger f, i.e. x = d^dagger, y = e,
// z = f^dagger (conjugation is an exact sign flip), so that lanes computing
// upper and lower terms side by side run one instruction stream (the
// cooperative kernel).
template <typename T, typename LT>
__device__ __forceinline__ Quat<T> staple_term(const LT& U, int mu, int nu, int p, uint32_t i,
                                               const int* hp, const int* hm, bool lower)
{
    const int q = p ^ 1;
    if (!lower) {
        const Quat<T> a = U.load(nu, q, i + hp[mu]);          // U_nu(x+mu)
        const Quat<T> b = U.load(mu, q, i + hp[nu]);          // U_mu(x+nu)
        const Quat<T> c = U.load(nu, p, i);                   // U_nu(x)
        return qmul_nd(qmul_nd(a, b), c);
    }
    const Quat<T> d = U.load(nu, p, i + hp[mu] + hm[nu]);     // U_nu(x+mu-nu)
    const Quat<T> e = U.load(mu, q, i + hm[nu]);              // U_mu(x-nu)
    const Quat<T> f = U.load(nu, q, i + hm[nu]);              // U_nu(x-nu)
    return qmul_nd(qmul_nd(qdag(d), e), qdag(f));
}

// (U: any link source with load(mu, parity, eo) -- global memory, or the
// distributed shared memory of a cluster)
template <typename T, int MU, bool PLAQ, typename LT>
__device__ __forceinline__ void staple_sum(const LT& U, const EoSite& s, uint32_t i, int p,
                                           Quat<T>& A, Quat<T>& P)
{
    int hp[4], hm[4];
    s.hops(hp, hm);
    if constexpr (std::is_same<T, double>::value) {
        Quat<T> sk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int nu = nu_of<MU>(k);
            sk[k] = qadd(staple_term<T>(U, MU, nu, p, i, hp, hm, false),
                         staple_term<T>(U, MU, nu, p, i, hp, hm, true));
        }
        const Quat<T> s01 = qadd(sk[0], sk[1]);
        A = qadd(s01, sk[2]);
        if (PLAQ) P = MU == 1 ? sk[0] : (MU == 2 ? s01 : A);
    } else {
        const int q = p ^ 1;
        const uint32_t e_pmu = i + hp[MU];
        A = {T(0), T(0), T(0), T(0)};
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
            // A += a b^dagger c^dagger + (e d)^dagger f, the sums fused into
            // the products' last steps
            A = qmul_dn_acc(qmul(e, d), f, qmul_nd_acc(qmul_nd(a, b), c, A));
            if (PLAQ && nu == MU - 1) P = A;
        }
    }
}

// The Kennedy-Pendleton trial on four uniforms:
// lambda^2 = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 alpha), delta = 2 lambda^2,
// accepted iff r4^2 <= 1 - lambda^2 (*lhs <= *rhs, compared by the caller,
// lane by lane for a pair).
template <typename V>
__device__ __forceinline__ void kp_eval(V r1, V r2, V r3, V r4, V inv2a, V* d, V* lhs, V* rhs)
{
    const V lam2 = mul_(neg_(fma_(Math<V>::cos2pi_sq(r2), Math<V>::ln_u01(r3),
                                  Math<V>::ln_u01(r1))), inv2a);
    *d = add_(lam2, lam2);
    *lhs = mul_(r4, r4);
    *rhs = add_(splat<V>(1.0f), neg_(lam2));
}

// One Kennedy-Pendleton trial from the four words of a Philox block.
template <typename T>
__device__ __forceinline__ bool kp_try(const U4& w, T inv2a, T* d)
{
    T lhs, rhs;
    kp_eval(u01<T>(w.x), u01<T>(w.y), u01<T>(w.z), u01<T>(w.w), inv2a, d, &lhs, &rhs);
    return lhs <= rhs;
}
// The same with the FP64 path's tables (unused in FP32).  FP64: kp_eval's
// operations, with the logarithms and cos(2 pi r2) table-driven
// (ln_u01_tab, sincospi_tab), their arguments read off the random bits.
template <typename T>
__device__ __forceinline__ bool kp_try(const U4& w, T inv2a, T* d, const double2* tab)
{
    (void)tab;
    return kp_try(w, inv2a, d);
}
template <>
__device__ __forceinline__ bool kp_try<double>(const U4& w, double inv2a, double* d,
                                               const double2* tab)
{
    double sn, c;  // cos(2 pi r2) from the table (the sine is not used)
    sincospi_tab(2u * (w.y >> 9) + 1u, 23, tab, &sn, &c);
    const double lam2 =
        mul_(neg_(fma_(mul_(c, c), ln_u01_tab(w.z, tab), ln_u01_tab(w.x, tab))), inv2a);
    *d = add_(lam2, lam2);
    const double r4 = u01d(w.w);
    return mul_(r4, r4) <= add_(1.0, neg_(lam2));
}

// One trial of Creutz's draw (small alpha): a0 from exp(alpha a0) by
// inversion, delta = -ln(1 - r1 qc) / alpha with qc = 1 - exp(-2 alpha),
// accepted with probability sqrt(1 - a0^2) = sqrt(delta (2 - delta)); the
// same trial blocks, r1 = word 0, r4 = word 3.
template <typename T>
__device__ __forceinline__ bool creutz_try(const U4& w, T qc, T inv2a, T* d)
{
    const T r1 = u01<T>(w.x), r4 = u01<T>(w.w);
    *d = mul_(neg_(Math<T>::log1p(mul_(neg_(r1), qc))), add_(inv2a, inv2a));
    return mul_(r4, r4) <= mul_(*d, add_(T(2), neg_(*d)));
}

template <typename T>
__device__ __forceinline__ T creutz_qc(T alpha)
{
    return neg_(Math<T>::expm1(mul_(T(-2), alpha)));
}

// The accepted draw X = (1 - delta, sqrt(delta (2 - delta)) n) with the
// direction n from the uniforms u1 (cos theta = 2 u1 - 1) and u2
// (phi = 2 pi u2), and the new link U = X A^dagger / |A|, renormalised.
// (cth = cos theta, sph / cph = sin / cos phi)
template <typename V>
__device__ __forceinline__ Quat<V> new_link_dir(V delta, V cth, V sph, V cph, const Quat<V>& A)
{
    const V one = splat<V>(1.0f);
    const V sth = Math<V>::sqrt_pos(mul_(add_(one, neg_(cth)), add_(one, cth)));
    const V vl = Math<V>::sqrt_pos(mul_(delta, add_(splat<V>(2.0f), neg_(delta))));
    const V vs = mul_(vl, sth);
    const Quat<V> X = {add_(one, neg_(delta)), mul_(vs, cph), mul_(vs, sph), mul_(vl, cth)};
    return qnormalise(qmul_nd(X, A));
}
template <typename V>
__device__ __forceinline__ Quat<V> new_link_u(V delta, V u1, V u2, const Quat<V>& A)
{
    const V cth = fma_(splat<V>(2.0f), u1, splat<V>(-1.0f));
    V sph, cph;
    Math<V>::sincos2pi(u2, &sph, &cph);
    return new_link_dir(delta, cth, sph, cph, A);
}

// the direction from the spare bits kd1, kd2 of the first trial block
template <typename T>
__device__ __forceinline__ Quat<T> new_link(T delta, uint32_t kd1, uint32_t kd2, const Quat<T>& A)
{
    return new_link_u(delta, u18<T>(kd1), u18<T>(kd2), A);
}
// FP64: cos theta = 2 u1 - 1 = (2 kd1 + 1 - 2^18) 2^-18 assembled exactly
// from the bits (new_link_u's value, without FP64 instructions)
__device__ __forceinline__ double dir_cth(uint32_t kd1)
{
    return exact_double((int32_t)(2u * kd1 + 1u) - (1 << 18), -18);
}
// with the FP64 path's tables (unused in FP32): FP64 takes phi's sine and
// cosine from sincospi_tab at 2 u2 = (2 kd2 + 1) 2^-18
template <typename T>
__device__ __forceinline__ Quat<T> new_link(T delta, uint32_t kd1, uint32_t kd2, const Quat<T>& A,
                                            const double2* tab)
{
    (void)tab;
    return new_link(delta, kd1, kd2, A);
}
template <>
__device__ __forceinline__ Quat<double> new_link<double>(double delta, uint32_t kd1, uint32_t kd2,
                                                         const Quat<double>& A, const double2* tab)
{
    double sph, cph;
    sincospi_tab(2u * kd2 + 1u, 18, tab, &sph, &cph);
    return new_link_dir(delta, dir_cth(kd1), sph, cph, A);
}

// the spare low 9 bits of the first trial's four words: two 18-bit uniforms
__device__ __forceinline__ uint32_t spare_bits_1(const U4& w) { return ((w.x & 511u) << 9) | (w.y & 511u); }
__device__ __forceinline__ uint32_t spare_bits_2(const U4& w) { return ((w.z & 511u) << 9) | (w.w & 511u); }

// Totals of one warp without any block barrier (a warp never waits for the
// block's slowest warp): trial counts go to spread per-lattice atomic slots
// (exact integers), cap hits to an atomic only when present, the
// plaquette to one partial per warp, summed later in a fixed order.
template <typename T, int MU, bool PLAQ, int NT>
__device__ __forceinline__ void warp_totals(const Ctx& ctx, int l, uint32_t blk0, uint32_t Vh,
                                            T plaq, uint32_t ntrial, uint32_t ncap)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wt = __reduce_add_sync(0xffffffffu, ntrial);
    const uint32_t wc = __reduce_add_sync(0xffffffffu, ncap);
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
        if (wc) {
            atomicAdd(&Dw->caps, (unsigned long long)wc);
            atomicOr(ctx.status, STATUS_CAP_HIT);
        }
    }
}

// One link update, U_mu(x) at storage index i of parity p in sweep sw: the
// staple sum, the Kennedy-Pendleton (or Creutz) draw and the new link *un.
// Returns the trials used (> 0), 0 for the Haar branch (alpha -> 0) or -1
// when the cap was hit (*un then undefined); *P is the staple part closing
// the plaquettes (PLAQ).
template <typename T, int MU, bool PLAQ, bool HYB, typename LT>
__device__ __forceinline__ int32_t update_link(const LT& U, const LatDesc& D, const EoSite& s,
                                               uint32_t i, int p, uint64_t sw, Quat<T>* un,
                                               Quat<T>* P)
{
    Quat<T> A;
    staple_sum<T, MU, PLAQ>(U, s, i, p, A, *P);

    // alpha = beta k and 1/(2 alpha) from one reciprocal square root of k^2
    const T k2 = qnorm2(A);
    const T rk = Math<T>::rsqrt(k2);
    const T beta = beta_of<T>(D);
    const T alpha = mul_(mul_(beta, k2), rk);
    const Stream st{(uint32_t)D.seed, (uint32_t)(D.seed >> 32), s.lex() * 4u + MU,
                    (uint32_t)sw, (uint32_t)(sw >> 32)};

    if (!(alpha >= alpha_haar<T>())) {
        // alpha -> 0 limit of the conditional law (zero staple or beta = 0)
        *un = haar_from<T>(st.draw(TAG_DIRECTION, 0));
        return 0;
    }
    const T inv2a = inv_two_alpha<T>(D, rk, beta);
    T delta = T(0);
    int32_t tr = -1;
    // trial 0 also carries the direction in the low 9 bits of its words
    const U4 w = st.draw(TAG_TRIAL, 0u);
    const uint32_t kd1 = spare_bits_1(w), kd2 = spare_bits_2(w);
    if (HYB && alpha < creutz_of<T>(D)) {
        const T qc = creutz_qc(alpha);
        for (int t = 0; t < KP_CAP; ++t) {
            if (creutz_try(t == 0 ? w : st.draw(TAG_TRIAL, (uint32_t)t), qc, inv2a, &delta)) {
                tr = t + 1;
                break;
            }
        }
    } else if (kp_try(w, inv2a, &delta, D.fp64_table)) {
        tr = 1;
    } else {
        for (int t = 1; t < KP_CAP; ++t) {
            if (kp_try(st.draw(TAG_TRIAL, (uint32_t)t), inv2a, &delta, D.fp64_table)) {
                tr = t + 1;
                break;
            }
        }
    }
    if (tr > 0) *un = new_link(delta, kd1, kd2, A, D.fp64_table);
    return tr;
}

// ---------------------------------------------------------------------------
// one link per thread
// ---------------------------------------------------------------------------
template <typename T, int MU, bool PLAQ, bool DBG, int NT, int MINB, bool SLAB, bool HYB>
__global__ void __launch_bounds__(NT, MINB)
hb_phase_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh;
    const uint32_t blk0 = first_block(ctx.phase_start, l);
    const uint32_t j = (blockIdx.x - blk0) * NT + threadIdx.x;  // traversal position
    const Links<T> U(ctx.links, D, ctx.status);

    T plaq = T(0);
    uint32_t ntrial = 0, ncap = 0;

    if (j < Vh) {
        uint32_t i = j;  // storage index of the site
        const EoSite s = SLAB ? EoSite::from_slab(D, j, p, &i) : EoSite(D, j, p);
        Quat<T> un, P;
        const int32_t tr = update_link<T, MU, PLAQ, HYB>(U, D, s, i, p, D.sweep, &un, &P);
        if (tr >= 0) {
            U.store(MU, p, i, un);
        } else {
            ncap = 1;
            if (PLAQ) un = U.load_rw(MU, p, i);
        }
        ntrial = tr > 0 ? (uint32_t)tr : (tr < 0 ? (uint32_t)KP_CAP : 0u);
        if (DBG) dbg[s.lex()] = tr;
        if (PLAQ) plaq = qretr(un, P);
    }
    warp_totals<T, MU, PLAQ, NT>(ctx, l, blk0, Vh, plaq, ntrial, ncap);
}

// ---------------------------------------------------------------------------
// neighbour rows staged in shared memory by bulk copies (FP32, Nh = 32)
// ---------------------------------------------------------------------------
// With Nh = 32 a warp's 32 consecutive storage indices are one row (fixed y,
// z, t, all x of one parity), and every one of the 18 neighbour sets of the
// row is again one row of some (direction, parity) plane: a y, z or t hop
// moves the whole row, an x hop rotates it within itself.  One lane copies
// the 18 rows (512 B each) into the warp's shared buffer with cp.async.bulk,
// completing on an mbarrier; each lane then reads its neighbour at the
// index (e mod 32) of its own neighbour e.
constexpr int STAGE_ROWS = 18;
constexpr uint32_t STAGE_ROW_BYTES = 32 * sizeof(float4);
constexpr uint32_t STAGE_WAIT_POLLS = 1u << 20;  // bounded wait (each poll waits a while)

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
// one contiguous global -> shared copy of `bytes` (16-byte aligned, a
// multiple of 16) completing on mbarrier m
__device__ __forceinline__ void bulk_to_shared(void* dst, const void* src, uint32_t bytes,
                                               uint64_t* m)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(m)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait for phase `parity` of m; false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity)
{
    for (uint32_t k = 0; k < STAGE_WAIT_POLLS; ++k)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

// storage index of load slot k (ν by ν: a, b, c, d, e, f as in staple_sum)
// and its (direction, parity) plane
template <int MU>
__device__ __forceinline__ uint32_t stage_site(int k, int p, uint32_t i, const int* hp,
                                               const int* hm, int* plane)
{
    const int nu = nu_of<MU>(k / 6), q = p ^ 1;
    switch (k % 6) {
    case 0: *plane = nu * 2 + q; return i + hp[MU];           // U_nu(x+mu)
    case 1: *plane = MU * 2 + q; return i + hp[nu];           // U_mu(x+nu)
    case 2: *plane = nu * 2 + p; return i;                    // U_nu(x)
    case 3: *plane = nu * 2 + p; return i + hp[MU] + hm[nu];  // U_nu(x+mu-nu)
    case 4: *plane = MU * 2 + q; return i + hm[nu];           // U_mu(x-nu)
    default: *plane = nu * 2 + q; return i + hm[nu];          // U_nu(x-nu)
    }
}

// lane 0 starts the 18 row copies of the warp's row (its own neighbours
// name the rows); the caller waits on m
template <int MU>
__device__ __forceinline__ void stage_issue(const Links<float>& U, int p, uint32_t i,
                                            const int* hp, const int* hm,
                                            float4 (*rows)[32], uint64_t* m)
{
    mbar_expect_tx(m, STAGE_ROWS * STAGE_ROW_BYTES);
#pragma unroll
    for (int k = 0; k < STAGE_ROWS; ++k) {
        int plane;
        const uint32_t e = stage_site<MU>(k, p, i, hp, hm, &plane);
        bulk_to_shared(rows[k], U.base + (size_t)plane * U.Vh + (e & ~31u), STAGE_ROW_BYTES, m);
    }
}

// staple_sum's FP32 arithmetic on the staged rows
template <int MU, bool PLAQ>
__device__ __forceinline__ void staple_sum_staged(const float4 (*rows)[32], int p, uint32_t i,
                                                  const int* hp, const int* hm, Quat<float>& A,
                                                  Quat<float>& P)
{
    auto ld = [&](int k) {
        int plane;
        const float4 v = rows[k][stage_site<MU>(k, p, i, hp, hm, &plane) & 31u];
        return Quat<float>{v.x, v.y, v.z, v.w};
    };
    A = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        const Quat<float> a = ld(6 * kk), b = ld(6 * kk + 1), c = ld(6 * kk + 2);
        const Quat<float> d = ld(6 * kk + 3), e = ld(6 * kk + 4), f = ld(6 * kk + 5);
        A = qmul_dn_acc(qmul(e, d), f, qmul_nd_acc(qmul_nd(a, b), c, A));
        if (PLAQ && nu_of<MU>(kk) == MU - 1) P = A;
    }
}

// ---------------------------------------------------------------------------
// R links per thread with a per-warp retry queue
// ---------------------------------------------------------------------------
// With one link per thread a warp repeats the trial loop until its last
// lane accepts, so a pass over Philox and the Kennedy-Pendleton test runs
// with most lanes idle.  Here a thread walks R links (R rounds of the
// block's NT consecutive positions); a link whose first trial is rejected
// leaves its staple and state in a per-warp queue in shared memory, and
// the warp retries queued links 32 at a time (one per lane) whenever 32
// are waiting, and once more after its last round.  Each link still takes
// the first accepted trial of its own sequence t = 0, 1, ..., so the links
// are bit-identical to those of the kernel above.
template <typename T, bool PLAQ, bool HYB>
struct RetryQueue {
    static constexpr int CAP = 64;  // < 32 held before a push of at most 32
    T a[4][CAP];                    // staple sum A
    T pl[PLAQ ? 4 : 1][PLAQ ? CAP : 1];  // its plaquette part P
    T inv2a[CAP];                   // 1 / (2 alpha)
    T qc[HYB ? CAP : 1];            // Creutz: 1 - exp(-2 alpha); 0: Kennedy-Pendleton
    uint32_t key[CAP];              // Philox counter word lex * 4 + mu
    uint32_t tk[CAP];               // next trial | first 18-bit direction word << 13
    uint32_t kd2[CAP];              // second 18-bit direction word
    uint32_t site[CAP];             // storage index
};

template <typename T, int MU, bool PLAQ, bool DBG, int NT, int MINB, bool SLAB, bool HYB, int R,
          bool PERSIST, bool STAGE = false>
__global__ void __launch_bounds__(NT, MINB)
hb_phase_queue_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    static_assert(KP_CAP <= (1 << 13), "trial index must fit 13 bits");
    static_assert(!STAGE || (std::is_same<T, float>::value && !SLAB),
                  "staged rows: FP32, plain traversal");
    using Queue = RetryQueue<T, PLAQ, HYB>;
    __shared__ Queue sq[NT / 32];
    __shared__ __align__(128) float4 srows[STAGE ? NT / 32 : 1][STAGE ? STAGE_ROWS : 1][32];
    __shared__ __align__(8) uint64_t smbar[NT / 32];

    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh;
    const uint32_t blk0 = first_block(ctx.phase_start, l);
    // tiles of NT R positions, one per block; a persistent shape's nb blocks
    // take them in grid-stride order (nb <= the tile count), and a block's
    // queue carries over from tile to tile
    const uint32_t nb = PERSIST ? __ldg(ctx.phase_start + l + 1) - blk0 : 0u;
    const uint32_t ntiles = PERSIST ? (Vh + NT * R - 1) / (NT * R) : 0u;
    uint32_t tile = blockIdx.x - blk0;
    const Links<T> U(ctx.links, D, ctx.status);
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    Queue& Q = sq[threadIdx.x >> 5];
    const T beta = beta_of<T>(D);
    const uint64_t sw = D.sweep;
    const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32);
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    const double2* const lnt = D.fp64_table;  // FP64's log and sin/cos tables

    T plaq = T(0);
    uint32_t ntrial = 0, ncap = 0;
    int cnt = 0;  // queued links (warp-uniform)
    // staged rows: lattices with one row per warp (Nh = 32); block-uniform
    const bool staged = STAGE && D.Nh == 32;
    uint64_t* mb = &smbar[threadIdx.x >> 5];
    uint32_t mphase = 0;
    if (staged) {
        if (lane == 0) mbar_init(mb, 1);
        __syncwarp();
    }

    // a final link: store, plaquette, trial count
    auto put = [&](uint32_t i, uint32_t key, const Quat<T>& un, const Quat<T>& P, int32_t tr) {
        U.store(MU, p, i, un);
        if (PLAQ) plaq = add_(plaq, qretr(un, P));
        ntrial += (uint32_t)tr;
        if (DBG) dbg[key >> 2] = tr;
    };
    auto push = [&](bool pend, const Quat<T>& A, const Quat<T>& P, T inv2a, T qc, uint32_t key,
                    uint32_t tk, uint32_t kd2, uint32_t i) {
        const uint32_t m = __ballot_sync(0xffffffffu, pend);
        if (pend) {
            const int e = cnt + __popc(m & below);
            Q.a[0][e] = A.a0; Q.a[1][e] = A.a1; Q.a[2][e] = A.a2; Q.a[3][e] = A.a3;
            if (PLAQ) { Q.pl[0][e] = P.a0; Q.pl[1][e] = P.a1; Q.pl[2][e] = P.a2; Q.pl[3][e] = P.a3; }
            Q.inv2a[e] = inv2a;
            if (HYB) Q.qc[e] = qc;
            Q.key[e] = key;
            Q.tk[e] = tk;
            Q.kd2[e] = kd2;
            Q.site[e] = i;
        }
        cnt += __popc(m);
        __syncwarp();
    };
    // one trial for each of the last n queued links, one link per lane
    auto retry = [&](int n) {
        const bool have = lane < n;
        Quat<T> A = {T(0), T(0), T(0), T(0)}, P = A;
        T inv2a = T(0), qc = T(0);
        uint32_t key = 0, tk = 0, kd2 = 0, i = 0;
        if (have) {
            const int e = cnt - n + lane;
            A = {Q.a[0][e], Q.a[1][e], Q.a[2][e], Q.a[3][e]};
            if (PLAQ) P = {Q.pl[0][e], Q.pl[1][e], Q.pl[2][e], Q.pl[3][e]};
            inv2a = Q.inv2a[e];
            if (HYB) qc = Q.qc[e];
            key = Q.key[e];
            tk = Q.tk[e];
            kd2 = Q.kd2[e];
            i = Q.site[e];
        }
        __syncwarp();
        cnt -= n;
        bool pend = false;
        if (have) {
            const uint32_t t = tk & 0x1FFFu, kd1 = tk >> 13;
            const Stream st{k0, k1, key, slo, shi};
            const U4 w = st.draw(TAG_TRIAL, t);
            T delta;
            const bool ok = (HYB && qc > T(0)) ? creutz_try(w, qc, inv2a, &delta)
                                               : kp_try(w, inv2a, &delta, lnt);
            if (ok) {
                put(i, key, new_link(delta, kd1, kd2, A, lnt), P, (int32_t)t + 1);
            } else if (t + 1 >= (uint32_t)KP_CAP) {
                // cap hit: the link keeps its value
                ncap += 1;
                ntrial += (uint32_t)KP_CAP;
                if (PLAQ) plaq = add_(plaq, qretr(U.load_rw(MU, p, i), P));
                if (DBG) dbg[key >> 2] = -1;
            } else {
                pend = true;
                tk = (t + 1) | (kd1 << 13);
            }
        }
        push(pend, A, P, inv2a, qc, key, tk, kd2, i);
    };

    do {
        const uint32_t j0 = tile * (NT * R) + threadIdx.x;
        for (int r = 0; r < R; ++r) {
            const uint32_t j = j0 + (uint32_t)r * NT;
            bool pend = false;
            Quat<T> A = {T(0), T(0), T(0), T(0)}, P = A;
            T inv2a = T(0), qc = T(0);
            uint32_t key = 0, tk = 0, kd2 = 0, i = j;
            if (j < Vh) {  // warp-uniform when staged (Vh is a multiple of 32 there)
                const EoSite s = SLAB ? EoSite::from_slab(D, j, p, &i) : EoSite(D, j, p);
                if constexpr (STAGE) {
                    if (staged) {
                        int hp[4], hm[4];
                        s.hops(hp, hm);
                        float4 (*rows)[32] = srows[threadIdx.x >> 5];
                        // the previous round's reads are done before new copies land
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) stage_issue<MU>(U, p, i, hp, hm, rows, mb);
                        const bool ok = mbar_wait(mb, mphase);
                        mphase ^= 1u;
                        if (!__all_sync(0xffffffffu, ok)) {
                            // give up the phase; let the copies in flight land first
                            if (lane == 0) atomicOr(ctx.status, STATUS_STAGE);
                            mbar_wait(mb, mphase ^ 1u);
                            return;
                        }
                        staple_sum_staged<MU, PLAQ>(rows, p, i, hp, hm, A, P);
                    } else {
                        staple_sum<T, MU, PLAQ>(U, s, i, p, A, P);
                    }
                } else {
                    staple_sum<T, MU, PLAQ>(U, s, i, p, A, P);
                }
                const T k2 = qnorm2(A);
                const T rk = Math<T>::rsqrt(k2);
                const T alpha = mul_(mul_(beta, k2), rk);
                key = s.lex() * 4u + MU;
                const Stream st{k0, k1, key, slo, shi};
                if (!(alpha >= alpha_haar<T>())) {
                    put(i, key, haar_from<T>(st.draw(TAG_DIRECTION, 0)), P, 0);
                } else {
                    inv2a = inv_two_alpha<T>(D, rk, beta);
                    const U4 w = st.draw(TAG_TRIAL, 0u);
                    const uint32_t kd1 = spare_bits_1(w);
                    kd2 = spare_bits_2(w);
                    T delta;
                    bool ok;
                    if (HYB && alpha < creutz_of<T>(D)) {
                        qc = creutz_qc(alpha);
                        ok = creutz_try(w, qc, inv2a, &delta);
                    } else {
                        ok = kp_try(w, inv2a, &delta, lnt);
                    }
                    if (ok) {
                        put(i, key, new_link(delta, kd1, kd2, A, lnt), P, 1);
                    } else {
                        pend = true;
                        tk = 1u | (kd1 << 13);
                    }
                }
            }
            push(pend, A, P, inv2a, qc, key, tk, kd2, i);
            while (cnt >= 32) retry(32);
        }
        tile += nb;
    } while (PERSIST && tile < ntiles);
    while (cnt > 0) retry(cnt < 32 ? cnt : 32);
    warp_totals<T, MU, PLAQ, NT>(ctx, l, blk0, Vh, plaq, ntrial, ncap);
}

// ---------------------------------------------------------------------------
// FP32 site pairs: two links per thread and round, packed arithmetic
// ---------------------------------------------------------------------------
// On a lattice stored as site pairs (t, t + Nt/2), one thread updates both
// links of a record at once: every load brings the two links' components
// side by side, and the staple products, the Kennedy-Pendleton arithmetic
// and the new links run as two-lane FFMA2/FMUL2/FADD2 instructions, with
// the hardware transcendentals and the Philox draws per lane.  Every lane
// performs exactly the scalar kernels' sequence of roundings, so the links
// are bit-identical to theirs.  A lane whose first trial is rejected joins
// the warp's retry queue as a single link; so does a lane of a pair whose
// other lane was rejected.

// Staple sums of the two links of pair q.  The lattice of pairs has t
// extent Nt/2; a t hop across its boundary lands in the other half of the
// lattice, i.e. in the OTHER lane of the neighbouring record, so for the
// pairs at t = Nt/2 - 1 (plus hop, tp) and t = 0 (minus hop, tm) those
// loads have their lanes exchanged.  EDGE selects that variant at compile
// time (a warp-uniform branch picks it): the other pairs pay nothing.
template <int MU, bool PLAQ, bool EDGE>
__device__ __forceinline__ void staple_sum_pair(const PairLinks& U, const EoSite& s, uint32_t i,
                                                int p, bool tp, bool tm, Quat<float2>& A,
                                                Quat<float2>& P)
{
    const int q = p ^ 1;
    int hp[4], hm[4];
    s.hops(hp, hm);
    const uint32_t e_pmu = i + hp[MU];
    const float2 z = splat<float2>(0.0f);
    A = {z, z, z, z};
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == MU) continue;
        const uint32_t e_pnu = i + hp[nu];
        const uint32_t e_mnu = i + hm[nu];
        const uint32_t e_pmu_mnu = i + hp[MU] + hm[nu];
        Quat<float2> a = U.load2(nu, q, e_pmu);      // U_nu(x+mu)
        Quat<float2> b = U.load2(MU, q, e_pnu);      // U_mu(x+nu)
        const Quat<float2> c = U.load2(nu, p, i);    // U_nu(x)
        Quat<float2> d = U.load2(nu, p, e_pmu_mnu);  // U_nu(x+mu-nu)
        Quat<float2> e = U.load2(MU, q, e_mnu);      // U_mu(x-nu)
        Quat<float2> f = U.load2(nu, q, e_mnu);      // U_nu(x-nu)
        if (EDGE) {
            const bool up_mu = MU == 3 && tp;  // x + mu crossed t = Nt/2
            const bool up_nu = nu == 3 && tp;  // x + nu crossed t = Nt/2
            const bool dn_nu = nu == 3 && tm;  // x - nu crossed t = 0
            if (up_mu) a = lanes_swapped(a);
            if (up_nu) b = lanes_swapped(b);
            if (up_mu || dn_nu) d = lanes_swapped(d);
            if (dn_nu) {
                e = lanes_swapped(e);
                f = lanes_swapped(f);
            }
        }
        A = qmul_dn_acc(qmul(e, d), f, qmul_nd_acc(qmul_nd(a, b), c, A));
        if (PLAQ && nu == MU - 1) P = A;
    }
}

template <int MU, bool PLAQ, bool DBG, int NT, int MINB, bool SLAB, bool HYB, int R, bool PERSIST>
__global__ void __launch_bounds__(NT, MINB)
hb_pair_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    using Queue = RetryQueue<float, PLAQ, HYB>;
    __shared__ Queue sq[NT / 32];

    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh, Vq = D.Vq;
    const uint32_t blk0 = first_block(ctx.phase_start, l);
    // tiles of NT R pairs, as the queued kernel's tiles of links
    const uint32_t nb = PERSIST ? __ldg(ctx.phase_start + l + 1) - blk0 : 0u;
    const uint32_t ntiles = PERSIST ? (Vq + NT * R - 1) / (NT * R) : 0u;
    uint32_t tile = blockIdx.x - blk0;
    const PairLinks U(ctx.links, D, ctx.status);
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    Queue& Q = sq[threadIdx.x >> 5];
    const float beta = D.beta_f, hib = D.half_inv_beta_f;
    const uint32_t nt2 = (uint32_t)D.Nt >> 1;
    const uint32_t lex_half = D.V >> 1;  // lex of lane 1 = lex of lane 0 + V/2
    const uint64_t sw = D.sweep;
    const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32);
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);

    float plaq = 0.0f;                          // single links (queue, lone lanes)
    float2 plaq2 = splat<float2>(0.0f);         // pairs, lane by lane
    uint32_t ntrial = 0, ncap = 0;
    int cnt = 0;  // queued links (warp-uniform)

    auto put = [&](uint32_t i, uint32_t key, const Quat<float>& un, const Quat<float>& P, int32_t tr) {
        U.store(MU, p, i, un);
        if (PLAQ) plaq = add_(plaq, qretr(un, P));
        ntrial += (uint32_t)tr;
        if (DBG) dbg[key >> 2] = tr;
    };
    auto push = [&](bool pend, const Quat<float>& A, const Quat<float>& P, float inv2a, float qc,
                    uint32_t key, uint32_t tk, uint32_t kd2, uint32_t i) {
        const uint32_t m = __ballot_sync(0xffffffffu, pend);
        if (pend) {
            const int e = cnt + __popc(m & below);
            Q.a[0][e] = A.a0; Q.a[1][e] = A.a1; Q.a[2][e] = A.a2; Q.a[3][e] = A.a3;
            if (PLAQ) { Q.pl[0][e] = P.a0; Q.pl[1][e] = P.a1; Q.pl[2][e] = P.a2; Q.pl[3][e] = P.a3; }
            Q.inv2a[e] = inv2a;
            if (HYB) Q.qc[e] = qc;
            Q.key[e] = key;
            Q.tk[e] = tk;
            Q.kd2[e] = kd2;
            Q.site[e] = i;
        }
        cnt += __popc(m);
        __syncwarp();
    };
    // one trial for each of the last n queued links, one link per lane
    auto retry = [&](int n) {
        const bool have = lane < n;
        Quat<float> A = {0.f, 0.f, 0.f, 0.f}, P = A;
        float inv2a = 0.f, qc = 0.f;
        uint32_t key = 0, tk = 0, kd2 = 0, i = 0;
        if (have) {
            const int e = cnt - n + lane;
            A = {Q.a[0][e], Q.a[1][e], Q.a[2][e], Q.a[3][e]};
            if (PLAQ) P = {Q.pl[0][e], Q.pl[1][e], Q.pl[2][e], Q.pl[3][e]};
            inv2a = Q.inv2a[e];
            if (HYB) qc = Q.qc[e];
            key = Q.key[e];
            tk = Q.tk[e];
            kd2 = Q.kd2[e];
            i = Q.site[e];
        }
        __syncwarp();
        cnt -= n;
        bool pend = false;
        if (have) {
            const uint32_t t = tk & 0x1FFFu, kd1 = tk >> 13;
            const Stream st{k0, k1, key, slo, shi};
            const U4 w = st.draw(TAG_TRIAL, t);
            float delta;
            const bool ok = (HYB && qc > 0.f) ? creutz_try(w, qc, inv2a, &delta)
                                              : kp_try(w, inv2a, &delta);
            if (ok) {
                put(i, key, new_link(delta, kd1, kd2, A), P, (int32_t)t + 1);
            } else if (t + 1 >= (uint32_t)KP_CAP) {
                // cap hit: the link keeps its value
                ncap += 1;
                ntrial += (uint32_t)KP_CAP;
                if (PLAQ) plaq = add_(plaq, qretr(U.load_rw(MU, p, i), P));
                if (DBG) dbg[key >> 2] = -1;
            } else {
                pend = true;
                tk = (t + 1) | (kd1 << 13);
            }
        }
        push(pend, A, P, inv2a, qc, key, tk, kd2, i);
    };

    do {
        const uint32_t j0 = tile * (NT * R) + threadIdx.x;
        for (int r = 0; r < R; ++r) {
            const uint32_t j = j0 + (uint32_t)r * NT;
            bool pend0 = false, pend1 = false;
            const float2 z = splat<float2>(0.0f);
            Quat<float2> A = {z, z, z, z}, P = A;
            float2 inv2a = z, qc = z;
            uint32_t key0 = 0, key1 = 0, tk0 = 0, tk1 = 0, kd20 = 0, kd21 = 0, i = j;
            if (j < Vq) {
                EoSite s = SLAB ? EoSite::from_slab_t(D, j, p, &i, nt2, D.div_nt2)
                                : EoSite(D, j, p);
                s.Nt = (int)nt2;  // hops wrap on the lattice of pairs
                const bool tp = s.c[3] == (int)nt2 - 1, tm = s.c[3] == 0;
                if (tp || tm) staple_sum_pair<MU, PLAQ, true>(U, s, i, p, tp, tm, A, P);
                else staple_sum_pair<MU, PLAQ, false>(U, s, i, p, false, false, A, P);
                const float2 k2 = qnorm2(A);
                const float2 rk = Math<float2>::rsqrt(k2);
                const float2 alpha = mul_(mul_(splat<float2>(beta), k2), rk);
                key0 = s.lex() * 4u + MU;
                key1 = (s.lex() + lex_half) * 4u + MU;
                const Stream st0{k0, k1, key0, slo, shi}, st1{k0, k1, key1, slo, shi};
                const bool haar0 = !(alpha.x >= alpha_haar<float>());
                const bool haar1 = !(alpha.y >= alpha_haar<float>());
                inv2a = mul_(rk, splat<float2>(hib));
                const U4 w0 = st0.draw(TAG_TRIAL, 0u), w1 = st1.draw(TAG_TRIAL, 0u);
                float2 delta, lhs, rhs;
                kp_eval(u01f2(w0.x, w1.x), u01f2(w0.y, w1.y), u01f2(w0.z, w1.z),
                        u01f2(w0.w, w1.w), inv2a, &delta, &lhs, &rhs);
                bool ok0 = lhs.x <= rhs.x, ok1 = lhs.y <= rhs.y;
                if (HYB) {
                    const float cb = D.creutz_below_f;
                    if (alpha.x < cb) {
                        qc.x = creutz_qc(alpha.x);
                        ok0 = creutz_try(w0, qc.x, inv2a.x, &delta.x);
                    }
                    if (alpha.y < cb) {
                        qc.y = creutz_qc(alpha.y);
                        ok1 = creutz_try(w1, qc.y, inv2a.y, &delta.y);
                    }
                }
                ok0 = ok0 && !haar0;
                ok1 = ok1 && !haar1;
                const uint32_t kd10 = spare_bits_1(w0), kd11 = spare_bits_1(w1);
                kd20 = spare_bits_2(w0);
                kd21 = spare_bits_2(w1);
                // both lanes' new links at once; a rejected lane's value is
                // never stored
                const Quat<float2> un =
                    new_link_u(delta, u18f2(kd10, kd11), u18f2(kd20, kd21), A);
                if (ok0 && ok1) {
                    U.store2(MU, p, i, un);
                    if (PLAQ) plaq2 = add_(plaq2, qretr(un, P));
                    ntrial += 2;
                    if (DBG) {
                        dbg[key0 >> 2] = 1;
                        dbg[key1 >> 2] = 1;
                    }
                } else {
                    if (ok0) put(i, key0, lane0(un), lane0(P), 1);
                    if (ok1) put(i + Vq, key1, lane1(un), lane1(P), 1);
                    if (haar0) put(i, key0, haar_from<float>(st0.draw(TAG_DIRECTION, 0)), lane0(P), 0);
                    if (haar1)
                        put(i + Vq, key1, haar_from<float>(st1.draw(TAG_DIRECTION, 0)), lane1(P), 0);
                    pend0 = !ok0 && !haar0;
                    pend1 = !ok1 && !haar1;
                    tk0 = 1u | (kd10 << 13);
                    tk1 = 1u | (kd11 << 13);
                }
            }
            push(pend0, lane0(A), lane0(P), inv2a.x, qc.x, key0, tk0, kd20, i);
            while (cnt >= 32) retry(32);
            push(pend1, lane1(A), lane1(P), inv2a.y, qc.y, key1, tk1, kd21, i + Vq);
            while (cnt >= 32) retry(32);
        }
        tile += nb;
    } while (PERSIST && tile < ntiles);
    while (cnt > 0) retry(cnt < 32 ? cnt : 32);
    if (PLAQ) plaq = add_(plaq, add_(plaq2.x, plaq2.y));
    warp_totals<float, MU, PLAQ, NT>(ctx, l, blk0, Vh, plaq, ntrial, ncap);
}

// ---------------------------------------------------------------------------
// FP64, G lanes per link: the cooperative kernel for small lattices
// ---------------------------------------------------------------------------
// On GB300 an FP64 warp instruction holds its SM sub-partition's FP64 unit
// for ~76 cycles, with one active lane as with 32, and a dependent one
// waits no longer than that; a small lattice (8^4: 2048 links per phase =
// 64 warps of one link per thread) leaves most sub-partitions without
// work.  Here G = 8 lanes share one link, and the phase takes about as long
// as one warp's stream of FP64 instructions, so the link's work is laid
// out for few instructions, not few lanes: lanes 0..5 compute the six
// staple terms at once (upper and lower in one stream), the sums follow the
// FP64 tree order above one component per lane, the lanes try
// Kennedy-Pendleton trials t0 .. t0 + 3 at once (one logarithm per lane)
// while two of them take the direction's cosine and sine in the trials'
// cospi stream, the two square roots of the new link share one stream, and
// lanes 0..3 form one component each of the final product.  The link takes the first
// accepted trial of its own sequence, as every other kernel does, and each
// value comes from the same operations as in the scalar kernels, so links
// and trial counts are bit-identical to theirs.
// x with its sign flipped where m has bit 63 set (an integer operation)
__device__ __forceinline__ double flip_sign(double x, uint64_t m)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
}
__device__ __forceinline__ Quat<double> qdag_if(const Quat<double>& q, uint64_t m)
{
    return {q.a0, flip_sign(q.a1, m), flip_sign(q.a2, m), flip_sign(q.a3, m)};
}

// the k-th of four values, by selects (no indexed local array)
template <typename V>
__device__ __forceinline__ V pick4(int k, V v0, V v1, V v2, V v3)
{
    return k == 0 ? v0 : (k == 1 ? v1 : (k == 2 ? v2 : v3));
}

// Component c of p q^dagger: qmul_nd's multiply and three fused
// multiply-adds for that component, in its order, on operands picked per
// lane, so four lanes form the four components in one stream with
// qmul_nd's bits.
__device__ __forceinline__ double qmul_nd_part(int c, const Quat<double>& p, const Quat<double>& q)
{
    constexpr uint64_t S = 0x8000000000000000ull;
    const double x0 = pick4(c, p.a0, p.a1, p.a2, p.a3);
    const double x1 = c == 0 ? p.a1 : p.a0;
    const double x2 = (c == 1 || c == 2) ? p.a3 : p.a2;
    const double x3 = pick4(c, p.a3, p.a2, p.a1, p.a1);
    const double y1 = flip_sign(pick4(c, q.a1, q.a1, q.a2, q.a3), c != 0 ? S : 0ull);
    const double y2 = flip_sign(pick4(c, q.a2, q.a2, q.a1, q.a1), (c & 1) ? S : 0ull);
    const double y3 = flip_sign(pick4(c, q.a3, q.a3, q.a3, q.a2), c == 2 ? S : 0ull);
    return fma_(x3, y3, fma_(x2, y2, fma_(x1, y1, mul_(x0, q.a0))));
}

template <typename T, int MU, bool PLAQ, bool DBG, int NT, int MINB, bool HYB, int G>
__global__ void __launch_bounds__(NT, MINB)
hb_phase_coop_kernel(Ctx ctx, int p, int32_t* __restrict__ dbg)
{
    static_assert(G == 8 && KP_CAP % G == 0, "eight lanes per link, whole trial groups");
    static_assert(std::is_same<T, double>::value, "the FP64 tree order of the staple");
    constexpr uint64_t SIGN = 0x8000000000000000ull;
    const int l = lattice_of_block(ctx.phase_start, ctx.n, blockIdx.x);
    const LatDesc& D = ctx.desc[l];
    const uint32_t Vh = D.Vh;
    const uint32_t blk0 = first_block(ctx.phase_start, l);
    const int lane = threadIdx.x & 31, g = lane & (G - 1), g0 = lane & ~(G - 1);
    const uint32_t j = (blockIdx.x - blk0) * (NT / G) + threadIdx.x / G;  // link position
    const bool act = j < Vh;  // uniform within the group
    const Links<T> U(ctx.links, D, ctx.status);
    // the per-call values, loaded up front (they are needed only after the
    // staple, and their loads then wait on nothing)
    const uint64_t sw = D.sweep, seed = D.seed;
    const T beta = beta_of<T>(D), hib = D.half_inv_beta;
    const double2* const lnt = D.fp64_table;

    Quat<T> term = {T(0), T(0), T(0), T(0)};
    uint32_t key = 0;
    const uint32_t i = j;
    if (act) {
        const EoSite s(D, j, p);
        int hp[4], hm[4];
        s.hops(hp, hm);
        key = s.lex() * 4u + MU;
        if (g < 6) {
            // lane 2k: the upper term of the k-th nu != mu, (a, b, c) =
            // (U_nu(x+mu), U_mu(x+nu), U_nu(x)); lane 2k+1: the lower one,
            // (d^dagger, e, f^dagger) = (U_nu(x+mu-nu)^dagger, U_mu(x-nu),
            // U_nu(x-nu)^dagger); each lane forms x y^dagger z^dagger
            const int nu = nu_of<MU>(g >> 1);
            const bool lower = (g & 1) != 0;
            const int q = p ^ 1;
            const int hpn = pick4(nu, hp[0], hp[1], hp[2], hp[3]);
            const int hmn = pick4(nu, hm[0], hm[1], hm[2], hm[3]);
            const uint64_t m = lower ? SIGN : 0ull;
            const Quat<T> x = qdag_if(U.load(nu, lower ? p : q, i + hp[MU] + (lower ? hmn : 0)), m);
            const Quat<T> y = U.load(MU, q, i + (lower ? hmn : hpn));
            const Quat<T> z = qdag_if(U.load(nu, lower ? q : p, lower ? i + hmn : i), m);
            term = qmul_nd(qmul_nd(x, y), z);
        }
    }
    // The tree s_k = up_k + lo_k, A = (s_0 + s_1) + s_2 one component per
    // lane: the terms go through shared memory, lane (kk, c) = (g >> 2, g & 3)
    // adds component c of s_kk and of s_2, lanes c and c + 4 swap theirs,
    // and every lane then holds component c of s_0, s_1, s_01 and A (four
    // additions in the stream instead of twelve).
    __shared__ double terms[NT / G][6][4];
    double* const tg6 = &terms[threadIdx.x / G][0][0];
    if (g < 6) {
        reinterpret_cast<double2*>(tg6 + 4 * g)[0] = make_double2(term.a0, term.a1);
        reinterpret_cast<double2*>(tg6 + 4 * g)[1] = make_double2(term.a2, term.a3);
    }
    __syncwarp();
    const int c = g & 3, kk = g >> 2;
    const T skc = add_(tg6[4 * (2 * kk) + c], tg6[4 * (2 * kk + 1) + c]);
    const T s2c = add_(tg6[16 + c], tg6[20 + c]);
    const T swp = __shfl_sync(0xffffffffu, skc, lane ^ 4);
    const T s0c = kk ? swp : skc, s1c = kk ? skc : swp;
    const T s01c = add_(s0c, s1c);
    const T Ac = add_(s01c, s2c);
    auto gather = [&](T v) -> Quat<T> {
        return {__shfl_sync(0xffffffffu, v, g0), __shfl_sync(0xffffffffu, v, g0 + 1),
                __shfl_sync(0xffffffffu, v, g0 + 2), __shfl_sync(0xffffffffu, v, g0 + 3)};
    };
    const Quat<T> A = gather(Ac);
    Quat<T> P = A;
    if (PLAQ && MU < 3) P = gather(MU == 1 ? s0c : s01c);

    const T k2 = qnorm2(A);
    const T rk = Math<T>::rsqrt(k2);
    const T alpha = mul_(mul_(beta, k2), rk);
    const Stream st{(uint32_t)seed, (uint32_t)(seed >> 32), key, (uint32_t)sw,
                    (uint32_t)(sw >> 32)};
    const bool haar = !(alpha >= alpha_haar<T>());
    const T inv2a = mul_(rk, hib);  // inv_two_alpha's product
    const bool creutz = HYB && alpha < creutz_of<T>(D);
    const T qc = creutz ? creutz_qc(alpha) : T(0);

    // Kennedy-Pendleton: lanes g and g + 4 share trial t0 + (g & 3), lane g
    // taking ln r1 and lane g + 4 ln r3, so each lane evaluates one logarithm
    // per pass and a pass tries four trials; in the first pass lanes 4 and 5
    // take the direction's cos(phi) and sin(phi), phi = 2 pi u2, from the
    // table's sine/cosine stream in place of the cos(2 pi r2) that only
    // lanes 0..3 use.
    // Creutz's draw needs one logarithm per trial, so there each of the eight
    // lanes tries its own (the direction still comes from lanes 4 and 5 of
    // the first pass).  Each group advances its own t0; the warp loops while
    // any link waits.
    const int stride = creutz ? G : G / 2;
    const int tg = creutz ? g : (g & 3);
    bool done = !act || haar;
    int32_t tr = -1;
    T delta = T(0), cph = T(0), sph = T(0);
    uint32_t kd1 = 0, kd2 = 0;
    int t0 = 0;
    for (int pass = 0;; ++pass) {
        if (!done && t0 >= KP_CAP) done = true;  // cap hit: tr stays -1
        if (!__any_sync(0xffffffffu, !done)) break;
        const U4 w = st.draw(TAG_TRIAL, (uint32_t)(t0 + tg));
        if (pass == 0) {  // the direction: spare bits of trial 0 (lane g0)
            kd1 = __shfl_sync(0xffffffffu, spare_bits_1(w), g0);
            kd2 = __shfl_sync(0xffffffffu, spare_bits_2(w), g0);
        }
        // kp_eval's pieces, with ln r3 from the partner lane (all lanes,
        // outside the branch: the shuffles need the whole warp)
        const T lnv = ln_u01_tab(g < 4 ? w.x : w.z, lnt);
        const T ln3 = __shfl_sync(0xffffffffu, lnv, lane ^ 4);
        // cos(2 pi r2) from the table; in the first pass lanes 4 and 5 take
        // the direction's cos phi and sin phi from the same stream
        const bool dir = pass == 0 && (g == 4 || g == 5);
        T sv, cv;
        sincospi_tab(dir ? 2u * kd2 + 1u : 2u * (w.y >> 9) + 1u, dir ? 18 : 23, lnt, &sv, &cv);
        const T dv = dir && g == 5 ? sv : cv;
        if (pass == 0) {
            cph = __shfl_sync(0xffffffffu, dv, g0 + 4);
            sph = __shfl_sync(0xffffffffu, dv, g0 + 5);
        }
        T d;
        bool ok;
        if (creutz) {
            ok = creutz_try(w, qc, inv2a, &d);
        } else {
            const T lam2 = mul_(neg_(fma_(mul_(cv, cv), ln3, lnv)), inv2a);
            d = add_(lam2, lam2);
            const T r4 = u01<T>(w.w);
            ok = g < 4 && mul_(r4, r4) <= add_(T(1), neg_(lam2));
        }
        ok = ok && !done;
        const uint32_t m = (__ballot_sync(0xffffffffu, ok) >> g0) & ((1u << G) - 1u);
        const int first = m ? __ffs(m) - 1 : 0;
        const T dfirst = __shfl_sync(0xffffffffu, d, g0 + first);
        if (!done && m) {
            done = true;
            tr = t0 + first + 1;
            delta = dfirst;
        }
        t0 += stride;
    }
    // the new link, new_link's arithmetic: lane 4 takes sin(theta) =
    // sqrt((1 - cth)(1 + cth)) and lane 5 |vector part| =
    // sqrt((delta + (-0)) (2 - delta)) in one stream
    const T one = T(1);
    const T cth = dir_cth(kd1);
    const bool l5 = g == 5;
    const T root = Math<T>::sqrt_pos(
        mul_(add_(l5 ? delta : one, l5 ? T(-0.0) : flip_sign(cth, SIGN)),
             add_(l5 ? T(2) : one, l5 ? flip_sign(delta, SIGN) : cth)));
    const T sth = __shfl_sync(0xffffffffu, root, g0 + 4);
    const T vl = __shfl_sync(0xffffffffu, root, g0 + 5);
    const T vs = mul_(vl, sth);
    const Quat<T> X = {add_(one, neg_(delta)), mul_(vs, cph), mul_(vs, sph), mul_(vl, cth)};
    // U = X A^dagger / |X A^dagger|: one component per lane, the norm on
    // every lane, the scaled components gathered on lane 0
    const T rc = qmul_nd_part(g & 3, X, A);
    const Quat<T> r = {__shfl_sync(0xffffffffu, rc, g0), __shfl_sync(0xffffffffu, rc, g0 + 1),
                       __shfl_sync(0xffffffffu, rc, g0 + 2), __shfl_sync(0xffffffffu, rc, g0 + 3)};
    const T uc = mul_(rc, rsqrt_t(qnorm2(r)));
    const Quat<T> unew = {__shfl_sync(0xffffffffu, uc, g0), __shfl_sync(0xffffffffu, uc, g0 + 1),
                          __shfl_sync(0xffffffffu, uc, g0 + 2), __shfl_sync(0xffffffffu, uc, g0 + 3)};
    T plaq = T(0);
    uint32_t ntrial = 0, ncap = 0;
    if (act && g == 0) {
        Quat<T> un = unew;
        if (haar) {
            un = haar_from<T>(st.draw(TAG_DIRECTION, 0));
            tr = 0;
        }
        if (tr >= 0) {
            U.store(MU, p, i, un);
        } else {
            ncap = 1;
            if (PLAQ) un = U.load_rw(MU, p, i);
        }
        ntrial = tr > 0 ? (uint32_t)tr : (tr < 0 ? (uint32_t)KP_CAP : 0u);
        if (DBG) dbg[key >> 2] = tr;
        if (PLAQ) plaq = qretr(un, P);
    }
    warp_totals<T, MU, PLAQ, NT>(ctx, l, blk0, Vh, plaq, ntrial, ncap);
}

// One launch shape (NT threads per block, at least MINB blocks per SM, R
// links -- or with PAIRS, R site pairs -- per thread, persistent or not) of
// the phase kernel; the grid covers ctx.phase_blocks blocks of NT R links
// or pairs (fewer, each walking several tiles, for a persistent shape on a
// single lattice).
template <typename T, int NT, int MINB, bool SLAB, int R = 1, bool PERSIST = false,
          bool PAIRS = false, int GROUP = 1, bool STAGE = false>
cudaError_t launch_phase_shape(const Ctx& c, int mu, int parity, bool plaq, int32_t* dbg,
                               bool hyb, cudaStream_t s)
{
    // the fused plaquette exists only in the odd phases with mu >= 1
    const bool pl = plaq && parity == 1 && mu >= 1;
    const dim3 grid(c.phase_blocks), block(NT);
#define SU2_K(MUV, PL, DB, H)                                                                   \
    if constexpr (GROUP > 1 && std::is_same<T, double>::value)                                  \
        hb_phase_coop_kernel<T, MUV, PL, DB, NT, MINB, H, GROUP><<<grid, block, 0, s>>>(        \
            c, parity, dbg);                                                                    \
    else if constexpr (PAIRS)                                                                   \
        hb_pair_kernel<MUV, PL, DB, NT, MINB, SLAB, H, R, PERSIST><<<grid, block, 0, s>>>(      \
            c, parity, dbg);                                                                    \
    else if constexpr (R == 1 && !PERSIST && !STAGE)                                            \
        hb_phase_kernel<T, MUV, PL, DB, NT, MINB, SLAB, H><<<grid, block, 0, s>>>(c, parity, dbg); \
    else                                                                                        \
        hb_phase_queue_kernel<T, MUV, PL, DB, NT, MINB, SLAB, H, R, PERSIST,                     \
                              STAGE && std::is_same<T, float>::value><<<grid, block, 0, s>>>(     \
            c, parity, dbg)
#define SU2_LAUNCH_H(MUV, H)                                    \
    do {                                                        \
        if (dbg) { SU2_K(MUV, false, true, H); }                \
        else if (pl) { SU2_K(MUV, (MUV > 0), false, H); }       \
        else { SU2_K(MUV, false, false, H); }                   \
    } while (0)
#define SU2_LAUNCH(MUV)                   \
    do {                                  \
        if (hyb) SU2_LAUNCH_H(MUV, true); \
        else SU2_LAUNCH_H(MUV, false);    \
    } while (0)
    switch (mu) {
    case 0: SU2_LAUNCH(0); break;
    case 1: SU2_LAUNCH(1); break;
    case 2: SU2_LAUNCH(2); break;
    default: SU2_LAUNCH(3); break;
    }
#undef SU2_LAUNCH
#undef SU2_LAUNCH_H
#undef SU2_K
    return cudaGetLastError();
}

}  // namespace su2
