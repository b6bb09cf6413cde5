// su2_device.cuh -- device building blocks of the SU(2) heat-bath library:
// quaternion algebra, the Philox4x32-10 counter generator, exact fast
// division by run-time constants and the even/odd site geometry.
//
// Conventions (the paper leaves them to its companion paper; they are fixed
// once for the whole library):
//   * a link is a unit quaternion (a0,a1,a2,a3) for U = a0 + i a.sigma,
//     1/2 Tr U = a0, det U = |a|^2;
//   * site (x,y,z,t), extents (Ns,Ns,Ns,Nt), lex = x + Ns(y + Ns(z + Ns t)),
//     parity (x+y+z+t) & 1, index inside one parity eo = lex >> 1;
//   * the random stream of link (lex, mu) in sweep s is Philox4x32-10 with
//     key (seed lo, seed hi) and counter (lex*4+mu, s lo, tag<<24 | trial,
//     s hi); tag 0 = Kennedy-Pendleton trial (its first block also feeds
//     the direction through the 9 low bits of each word), 1 = Haar draw,
//     2 = hot start, 3 = random gauge transformation.  The stream therefore
//     never depends on launch shape, batch position or graph replay.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace su2 {

// --------------------------------------------------------------------------
// arithmetic with every rounding written out
// --------------------------------------------------------------------------
// Each multiply, add and fused multiply-add of the update is an explicit
// round-to-nearest intrinsic, so the compiler never contracts or
// re-associates them.  The same sequence then runs on one value (float,
// double) or on two FP32 lanes at once (float2: Blackwell's packed
// FFMA2/FMUL2/FADD2), and the two give identical bits in every lane.
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 mul_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ double neg_(double a) { return -a; }
// packed negation: one FMUL2 by -1 (exact) instead of one instruction per lane
__device__ __forceinline__ float2 neg_(float2 a) { return __fmul2_rn(a, make_float2(-1.0f, -1.0f)); }
// a constant in every lane
template <typename V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ double splat<double>(float c) { return (double)c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }

// --------------------------------------------------------------------------
// quaternions (V = float, double, or float2 for two links at once)
// --------------------------------------------------------------------------
template <typename T>
struct Quat {
    T a0, a1, a2, a3;
};

template <typename T>
__device__ __forceinline__ Quat<T> qadd(const Quat<T>& p, const Quat<T>& q)
{
    return {add_(p.a0, q.a0), add_(p.a1, q.a1), add_(p.a2, q.a2), add_(p.a3, q.a3)};
}

// The products are written so that every term enters with a plus sign,
// the minus signs carried by three negated components of one operand:
// negation is free in scalar instructions but costs an instruction on a
// packed pair, so each product negates no more than three values.

// p q  for U = a0 + i a.sigma:  (p0 q0 - p.q,  p0 q + q0 p - p x q);
// negated: the vector part of q
template <typename T>
__device__ __forceinline__ Quat<T> qmul(const Quat<T>& p, const Quat<T>& q)
{
    const T n1 = neg_(q.a1), n2 = neg_(q.a2), n3 = neg_(q.a3);
    Quat<T> r;
    r.a0 = fma_(p.a3, n3, fma_(p.a2, n2, fma_(p.a1, n1, mul_(p.a0, q.a0))));
    r.a1 = fma_(p.a2, n3, fma_(p.a3, q.a2, fma_(p.a0, q.a1, mul_(p.a1, q.a0))));
    r.a2 = fma_(p.a1, q.a3, fma_(p.a3, n1, fma_(p.a0, q.a2, mul_(p.a2, q.a0))));
    r.a3 = fma_(p.a1, n2, fma_(p.a2, q.a1, fma_(p.a0, q.a3, mul_(p.a3, q.a0))));
    return r;
}

template <typename T>
__device__ __forceinline__ Quat<T> qdag(const Quat<T>& p)
{
    return {p.a0, neg_(p.a1), neg_(p.a2), neg_(p.a3)};
}

// p q^dagger; negated: the vector part of q
template <typename T>
__device__ __forceinline__ Quat<T> qmul_nd(const Quat<T>& p, const Quat<T>& q)
{
    const T n1 = neg_(q.a1), n2 = neg_(q.a2), n3 = neg_(q.a3);
    Quat<T> r;
    r.a0 = fma_(p.a3, q.a3, fma_(p.a2, q.a2, fma_(p.a1, q.a1, mul_(p.a0, q.a0))));
    r.a1 = fma_(p.a2, q.a3, fma_(p.a3, n2, fma_(p.a0, n1, mul_(p.a1, q.a0))));
    r.a2 = fma_(p.a1, n3, fma_(p.a3, q.a1, fma_(p.a0, n2, mul_(p.a2, q.a0))));
    r.a3 = fma_(p.a1, q.a2, fma_(p.a2, n1, fma_(p.a0, n3, mul_(p.a3, q.a0))));
    return r;
}

// p^dagger q; negated: the vector part of p
template <typename T>
__device__ __forceinline__ Quat<T> qmul_dn(const Quat<T>& p, const Quat<T>& q)
{
    const T n1 = neg_(p.a1), n2 = neg_(p.a2), n3 = neg_(p.a3);
    Quat<T> r;
    r.a0 = fma_(p.a3, q.a3, fma_(p.a2, q.a2, fma_(p.a1, q.a1, mul_(p.a0, q.a0))));
    r.a1 = fma_(n3, q.a2, fma_(p.a2, q.a3, fma_(n1, q.a0, mul_(p.a0, q.a1))));
    r.a2 = fma_(n1, q.a3, fma_(p.a3, q.a1, fma_(n2, q.a0, mul_(p.a0, q.a2))));
    r.a3 = fma_(n2, q.a1, fma_(p.a1, q.a2, fma_(n3, q.a0, mul_(p.a0, q.a3))));
    return r;
}

// acc + p q^dagger and acc + p^dagger q: the sum folded into the first
// multiply of each component (one rounding fewer, no separate additions)
template <typename T>
__device__ __forceinline__ Quat<T> qmul_nd_acc(const Quat<T>& p, const Quat<T>& q, const Quat<T>& acc)
{
    const T n1 = neg_(q.a1), n2 = neg_(q.a2), n3 = neg_(q.a3);
    Quat<T> r;
    r.a0 = fma_(p.a3, q.a3, fma_(p.a2, q.a2, fma_(p.a1, q.a1, fma_(p.a0, q.a0, acc.a0))));
    r.a1 = fma_(p.a2, q.a3, fma_(p.a3, n2, fma_(p.a0, n1, fma_(p.a1, q.a0, acc.a1))));
    r.a2 = fma_(p.a1, n3, fma_(p.a3, q.a1, fma_(p.a0, n2, fma_(p.a2, q.a0, acc.a2))));
    r.a3 = fma_(p.a1, q.a2, fma_(p.a2, n1, fma_(p.a0, n3, fma_(p.a3, q.a0, acc.a3))));
    return r;
}
template <typename T>
__device__ __forceinline__ Quat<T> qmul_dn_acc(const Quat<T>& p, const Quat<T>& q, const Quat<T>& acc)
{
    const T n1 = neg_(p.a1), n2 = neg_(p.a2), n3 = neg_(p.a3);
    Quat<T> r;
    r.a0 = fma_(p.a3, q.a3, fma_(p.a2, q.a2, fma_(p.a1, q.a1, fma_(p.a0, q.a0, acc.a0))));
    r.a1 = fma_(n3, q.a2, fma_(p.a2, q.a3, fma_(n1, q.a0, fma_(p.a0, q.a1, acc.a1))));
    r.a2 = fma_(n1, q.a3, fma_(p.a3, q.a1, fma_(n2, q.a0, fma_(p.a0, q.a2, acc.a2))));
    r.a3 = fma_(n2, q.a1, fma_(p.a1, q.a2, fma_(n3, q.a0, fma_(p.a0, q.a3, acc.a3))));
    return r;
}

// 1/2 Re Tr (p q) = p0 q0 - p.q
template <typename T>
__device__ __forceinline__ T qretr(const Quat<T>& p, const Quat<T>& q)
{
    return fma_(p.a3, neg_(q.a3), fma_(p.a2, neg_(q.a2), fma_(p.a1, neg_(q.a1), mul_(p.a0, q.a0))));
}

template <typename T>
__device__ __forceinline__ T qnorm2(const Quat<T>& p)
{
    return fma_(p.a3, p.a3, fma_(p.a2, p.a2, fma_(p.a1, p.a1, mul_(p.a0, p.a0))));
}

// lane 0 / lane 1 of a pair of quaternions
__device__ __forceinline__ Quat<float> lane0(const Quat<float2>& q)
{
    return {q.a0.x, q.a1.x, q.a2.x, q.a3.x};
}
__device__ __forceinline__ Quat<float> lane1(const Quat<float2>& q)
{
    return {q.a0.y, q.a1.y, q.a2.y, q.a3.y};
}
// the pair with its two lanes exchanged
__device__ __forceinline__ Quat<float2> lanes_swapped(const Quat<float2>& q)
{
    return {make_float2(q.a0.y, q.a0.x), make_float2(q.a1.y, q.a1.x),
            make_float2(q.a2.y, q.a2.x), make_float2(q.a3.y, q.a3.x)};
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return ::rsqrt(x); }

__device__ __forceinline__ float2 rsqrt_t(float2 x) { return make_float2(rsqrtf(x.x), rsqrtf(x.y)); }

template <typename T>
__device__ __forceinline__ Quat<T> qnormalise(const Quat<T>& p)
{
    const T s = rsqrt_t(qnorm2(p));
    return {mul_(p.a0, s), mul_(p.a1, s), mul_(p.a2, s), mul_(p.a3, s)};
}

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
// --------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

enum : uint32_t { TAG_TRIAL = 0u, TAG_DIRECTION = 1u, TAG_HOT = 2u, TAG_GAUGE = 3u };

struct Stream {
    uint32_t k0, k1;     // key
    uint32_t link;       // lex*4 + mu
    uint32_t s_lo, s_hi; // sweep
    __device__ __forceinline__ U4 draw(uint32_t tag, uint32_t trial) const
    {
        return philox4x32_10(U4{link, s_lo, (tag << 24) | trial, s_hi}, k0, k1);
    }
};

// uniform in (0,1): ((w >> 9) + 0.5) 2^-23, exact in float and double.
// FP32: the top 23 bits as the leading mantissa bits of a number in [1,2)
// give 1 + k 2^-23; subtracting 1 - 2^-24 leaves (2k + 1) 2^-24 exactly
// (Sterbenz).  FP64: the same value assembled from its bits (exact_double).
__device__ __forceinline__ float u01_bits(uint32_t w)  // 1 + k 2^-23
{
    return __int_as_float((int)((w >> 9) | 0x3F800000u));
}
__device__ __forceinline__ float u01f(uint32_t w)
{
    return add_(u01_bits(w), -0.99999994039535522f);
}
// two uniforms at once (one packed subtraction, the same bits per lane)
__device__ __forceinline__ float2 u01f2(uint32_t wa, uint32_t wb)
{
    return add_(make_float2(u01_bits(wa), u01_bits(wb)), splat<float2>(-0.99999994039535522f));
}
// m 2^e as a double, for an integer 0 < |m| < 2^31, assembled from its bits
// with integer operations only (the value is exact): on GB300 an FP64
// instruction holds its SM sub-partition's FP64 unit for ~76 cycles, so the
// uniforms of the FP64 path cost none
__device__ __forceinline__ double exact_double(int32_t m, int e)
{
    const uint32_t a = (uint32_t)(m < 0 ? -m : m);
    const int p = 31 - __clz((int)a);  // position of the leading bit
    const uint64_t f = ((uint64_t)a << (52 - p)) & 0x000FFFFFFFFFFFFFull;
    const uint32_t hi = (m < 0 ? 0x80000000u : 0u) | ((uint32_t)(1023 + p + e) << 20) |
                        (uint32_t)(f >> 32);
    return __hiloint2double((int)hi, (int)(uint32_t)f);
}
// ((w >> 9) + 1/2) 2^-23 = (2 (w >> 9) + 1) 2^-24
__device__ __forceinline__ double u01d(uint32_t w)
{
    return exact_double((int32_t)(2u * (w >> 9) + 1u), -24);
}
// uniform in (0,1) from an 18-bit integer k: (k + 0.5) 2^-18, exact
__device__ __forceinline__ float u18_bits(uint32_t k)
{
    return __int_as_float((int)(0x3F800000u | (k << 5)));
}
__device__ __forceinline__ float u18f(uint32_t k)
{
    return add_(u18_bits(k), -0.9999980926513671875f);
}
__device__ __forceinline__ float2 u18f2(uint32_t ka, uint32_t kb)
{
    return add_(make_float2(u18_bits(ka), u18_bits(kb)), splat<float2>(-0.9999980926513671875f));
}
// (k + 1/2) 2^-18 = (2 k + 1) 2^-19
__device__ __forceinline__ double u18d(uint32_t k)
{
    return exact_double((int32_t)(2u * k + 1u), -19);
}
template <typename T> __device__ __forceinline__ T u18(uint32_t k);
template <> __device__ __forceinline__ float u18<float>(uint32_t k) { return u18f(k); }
template <> __device__ __forceinline__ double u18<double>(uint32_t k) { return u18d(k); }

template <typename T> __device__ __forceinline__ T u01(uint32_t w);
template <> __device__ __forceinline__ float u01<float>(uint32_t w) { return u01f(w); }
template <> __device__ __forceinline__ double u01<double>(uint32_t w) { return u01d(w); }

// math wrappers with one spelling for both precisions
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }
__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// Haar element of SU(2) from one Philox block: Box-Muller on (w0,w1) and
// (w2,w3) gives four normals, normalised onto S^3.
template <typename T>
__device__ __forceinline__ Quat<T> haar_from(U4 w)
{
    const T u0 = u01<T>(w.x), u1 = u01<T>(w.y), u2 = u01<T>(w.z), u3 = u01<T>(w.w);
    const T r0 = sqrt_t(mul_(T(-2), log_t(u0)));
    const T r1 = sqrt_t(mul_(T(-2), log_t(u2)));
    T s0, c0, s1, c1;
    sincospi_t(mul_(T(2), u1), &s0, &c0);
    sincospi_t(mul_(T(2), u3), &s1, &c1);
    return qnormalise(Quat<T>{mul_(r0, c0), mul_(r0, s0), mul_(r1, c1), mul_(r1, s1)});
}

// --------------------------------------------------------------------------
// exact division of 0 <= n < 2^31 by a run-time constant d >= 1
// (multiply-high with a rounded-up reciprocal: Granlund & Montgomery 1994)
// --------------------------------------------------------------------------
struct FastDiv {
    uint32_t d, m, s;
};

__host__ __device__ __forceinline__ uint32_t umulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    // m = floor(2^32 (2^s - d) / d) + 1
    f.m = (uint32_t)((((1ull << s) - d) << 32) / d + 1);
    return f;
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    return (umulhi32(n, f.m) + n) >> f.s;
}

}  // namespace su2
