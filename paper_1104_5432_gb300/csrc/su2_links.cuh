// su2_links.cuh -- typed access to one lattice's links in the even/odd
// structure-of-arrays layout, and the decomposition of an even/odd index
// into coordinates and neighbours.
#pragma once
#include "su2_internal.h"

namespace su2 {

// Bounds-checked builds (-DSU2_CHECK_BOUNDS, for testing): every link
// access checks its even/odd index and direction; a bad one sets
// STATUS_BOUNDS in the handle's status word (reported as SU2_E_BOUNDS by
// the next synchronising call), reads link 0 instead and skips a store.
// Ordinary builds compile the checks away.
struct LinkCheck {
#ifdef SU2_CHECK_BOUNDS
    uint32_t* status;
    uint32_t Vh;
    __device__ __forceinline__ bool ok(int mu, int p, uint32_t eo) const
    {
        const bool good = eo < Vh && mu >= 0 && mu < 4 && (p == 0 || p == 1);
        if (!good && status) atomicOr(status, STATUS_BOUNDS);
        return good;
    }
#else
    __device__ __forceinline__ bool ok(int, int, uint32_t) const { return true; }
#endif
};

template <typename T> struct Links;

// FP32: float4 U[mu][parity][eo]
template <> struct Links<float> {
    float4* base;
    uint32_t Vh;
    LinkCheck chk;
    __device__ __forceinline__ Links(void* links, const LatDesc& d, uint32_t* status = nullptr)
        : base(reinterpret_cast<float4*>(static_cast<char*>(links) + d.link_off)), Vh(d.Vh)
    {
#ifdef SU2_CHECK_BOUNDS
        chk = {status, d.Vh};
#else
        (void)status;
#endif
    }
    __device__ __forceinline__ size_t idx(int mu, int p, uint32_t eo) const
    {
        return chk.ok(mu, p, eo) ? size_t(mu * 2 + p) * Vh + eo : 0;
    }
    __device__ __forceinline__ Quat<float> load(int mu, int p, uint32_t eo) const
    {
        const float4 v = __ldg(base + idx(mu, p, eo));
        return {v.x, v.y, v.z, v.w};
    }
    __device__ __forceinline__ Quat<float> load_rw(int mu, int p, uint32_t eo) const
    {
        const float4 v = base[idx(mu, p, eo)];
        return {v.x, v.y, v.z, v.w};
    }
    __device__ __forceinline__ void store(int mu, int p, uint32_t eo, const Quat<float>& q) const
    {
        if (chk.ok(mu, p, eo)) base[size_t(mu * 2 + p) * Vh + eo] = make_float4(q.a0, q.a1, q.a2, q.a3);
    }
};

// FP64: double2 U[mu][parity][plane][eo]
template <> struct Links<double> {
    double2* base;
    uint32_t Vh;
    LinkCheck chk;
    __device__ __forceinline__ Links(void* links, const LatDesc& d, uint32_t* status = nullptr)
        : base(reinterpret_cast<double2*>(static_cast<char*>(links) + d.link_off)), Vh(d.Vh)
    {
#ifdef SU2_CHECK_BOUNDS
        chk = {status, d.Vh};
#else
        (void)status;
#endif
    }
    __device__ __forceinline__ size_t idx(int mu, int p, int plane, uint32_t eo) const
    {
        return chk.ok(mu, p, eo) ? size_t((mu * 2 + p) * 2 + plane) * Vh + eo : 0;
    }
    __device__ __forceinline__ Quat<double> load(int mu, int p, uint32_t eo) const
    {
        const double2 lo = __ldg(base + idx(mu, p, 0, eo));
        const double2 hi = __ldg(base + idx(mu, p, 1, eo));
        return {lo.x, lo.y, hi.x, hi.y};
    }
    __device__ __forceinline__ Quat<double> load_rw(int mu, int p, uint32_t eo) const
    {
        const double2 lo = base[idx(mu, p, 0, eo)];
        const double2 hi = base[idx(mu, p, 1, eo)];
        return {lo.x, lo.y, hi.x, hi.y};
    }
    __device__ __forceinline__ void store(int mu, int p, uint32_t eo, const Quat<double>& q) const
    {
        if (!chk.ok(mu, p, eo)) return;
        base[size_t((mu * 2 + p) * 2 + 0) * Vh + eo] = make_double2(q.a0, q.a1);
        base[size_t((mu * 2 + p) * 2 + 1) * Vh + eo] = make_double2(q.a2, q.a3);
    }
};

// FP32 site pairs: float4 U[mu][parity][q][2], record q holding the sites
// eo = q (lane 0) and eo = q + Vq (lane 1) as (a0, a0', a1, a1'),
// (a2, a2', a3, a3').  Pair access for the paired phase kernel, single-site
// access (two floats of each half of the record) for everything else.
struct PairLinks {
    float4* base;
    uint32_t Vh, Vq;
    LinkCheck chk;
    __device__ __forceinline__ PairLinks(void* links, const LatDesc& d, uint32_t* status = nullptr)
        : base(reinterpret_cast<float4*>(static_cast<char*>(links) + d.link_off)), Vh(d.Vh),
          Vq(d.Vq)
    {
#ifdef SU2_CHECK_BOUNDS
        chk = {status, d.Vq};
#else
        (void)status;
#endif
    }
    // float4 index of the first half of record q
    __device__ __forceinline__ size_t ridx(int mu, int p, uint32_t q) const
    {
        return chk.ok(mu, p, q) ? size_t(mu * 2 + p) * Vh + 2 * (size_t)q : 0;
    }
    __device__ __forceinline__ Quat<float2> load2(int mu, int p, uint32_t q) const
    {
        const size_t i = ridx(mu, p, q);
        const float4 lo = __ldg(base + i), hi = __ldg(base + i + 1);
        return {make_float2(lo.x, lo.y), make_float2(lo.z, lo.w), make_float2(hi.x, hi.y),
                make_float2(hi.z, hi.w)};
    }
    __device__ __forceinline__ void store2(int mu, int p, uint32_t q, const Quat<float2>& u) const
    {
        if (!chk.ok(mu, p, q)) return;
        const size_t i = size_t(mu * 2 + p) * Vh + 2 * (size_t)q;
        base[i] = make_float4(u.a0.x, u.a0.y, u.a1.x, u.a1.y);
        base[i + 1] = make_float4(u.a2.x, u.a2.y, u.a3.x, u.a3.y);
    }
    // one site eo (either lane): the floats at lane, 2 + lane, 4 + lane, 6 + lane
    __device__ __forceinline__ const float* site(int mu, int p, uint32_t eo) const
    {
        const uint32_t h = eo >= Vq ? 1u : 0u;
        return reinterpret_cast<const float*>(base + ridx(mu, p, eo - h * Vq)) + h;
    }
    __device__ __forceinline__ Quat<float> load(int mu, int p, uint32_t eo) const
    {
        const float* f = site(mu, p, eo);
        return {__ldg(f), __ldg(f + 2), __ldg(f + 4), __ldg(f + 6)};
    }
    __device__ __forceinline__ Quat<float> load_rw(int mu, int p, uint32_t eo) const
    {
        const float* f = site(mu, p, eo);
        return {f[0], f[2], f[4], f[6]};
    }
    __device__ __forceinline__ void store(int mu, int p, uint32_t eo, const Quat<float>& a) const
    {
        const uint32_t h = eo >= Vq ? 1u : 0u;
        if (!chk.ok(mu, p, eo - h * Vq)) return;
        float* f = reinterpret_cast<float*>(base + size_t(mu * 2 + p) * Vh + 2 * (size_t)(eo - h * Vq)) + h;
        f[0] = a.a0;
        f[2] = a.a1;
        f[4] = a.a2;
        f[6] = a.a3;
    }
};

// Single-site access in whichever layout the lattice uses (the kernels
// outside the heat-bath phases: start, layout conversion, measurements).
template <typename T> struct AnyLinks;
template <> struct AnyLinks<double> : Links<double> {
    __device__ __forceinline__ AnyLinks(void* links, const LatDesc& d, uint32_t* status = nullptr)
        : Links<double>(links, d, status) {}
};
template <> struct AnyLinks<float> {
    Links<float> plain;
    PairLinks pairs;
    bool paired;
    __device__ __forceinline__ AnyLinks(void* links, const LatDesc& d, uint32_t* status = nullptr)
        : plain(links, d, status), pairs(links, d, status), paired(d.paired != 0) {}
    __device__ __forceinline__ Quat<float> load(int mu, int p, uint32_t eo) const
    {
        return paired ? pairs.load(mu, p, eo) : plain.load(mu, p, eo);
    }
    __device__ __forceinline__ Quat<float> load_rw(int mu, int p, uint32_t eo) const
    {
        return paired ? pairs.load_rw(mu, p, eo) : plain.load_rw(mu, p, eo);
    }
    __device__ __forceinline__ void store(int mu, int p, uint32_t eo, const Quat<float>& a) const
    {
        if (paired) pairs.store(mu, p, eo, a);
        else plain.store(mu, p, eo, a);
    }
};

// Coordinates of the site with index eo inside parity p.
struct EoSite {
    int c[4];        // x, y, z, t
    int Ns, Nt;
    uint32_t Nh;
    uint32_t r;      // row = y + Ns (z + Ns t);  eo = x/2 + Nh r;  lex = x + Ns r

    __device__ __forceinline__ EoSite(const LatDesc& d, uint32_t eo, int p)
    {
        Ns = d.Ns;
        Nt = d.Nt;
        Nh = (uint32_t)d.Nh;
        r = fdiv(eo, d.div_nh);
        const uint32_t xh = eo - r * Nh;
        const uint32_t q = fdiv(r, d.div_ns);
        const uint32_t y = r - q * (uint32_t)Ns;
        const uint32_t t = fdiv(q, d.div_ns);
        const uint32_t z = q - t * (uint32_t)Ns;
        c[1] = (int)y;
        c[2] = (int)z;
        c[3] = (int)t;
        c[0] = (int)(2 * xh) + ((p + c[1] + c[2] + c[3]) & 1);
    }

    // The site visited at traversal position j of a phase when the lattice is
    // walked in d.ysplit slabs of y (slab outermost, then t, z, y inside the
    // slab, x fastest).  Slabs keep the +-t neighbours of the sites in
    // flight within a window of Nh (Ns/ysplit) Ns sites, so that window
    // stays in L2 on large lattices.  *eo gets the storage index.
    __device__ __forceinline__ static EoSite from_slab(const LatDesc& d, uint32_t j, int p,
                                                       uint32_t* eo)
    {
        return from_slab_t(d, j, p, eo, (uint32_t)d.Nt, d.div_nt);
    }
    // the same walk over a lattice of t extent nt (the site pairs: Nt / 2)
    __device__ __forceinline__ static EoSite from_slab_t(const LatDesc& d, uint32_t j, int p,
                                                         uint32_t* eo, uint32_t nt,
                                                         const FastDiv& div_t)
    {
        const uint32_t r = fdiv(j, d.div_nh);
        const uint32_t xh = j - r * (uint32_t)d.Nh;
        const uint32_t r2 = fdiv(r, d.div_ny);
        const uint32_t yl = r - r2 * (uint32_t)d.Ny;
        const uint32_t r3 = fdiv(r2, d.div_ns);
        const uint32_t z = r2 - r3 * (uint32_t)d.Ns;
        const uint32_t ys = fdiv(r3, div_t);
        const uint32_t t = r3 - ys * nt;
        const uint32_t y = ys * (uint32_t)d.Ny + yl;
        *eo = xh + (uint32_t)d.Nh * (y + (uint32_t)d.Ns * (z + (uint32_t)d.Ns * t));
        return EoSite(d, *eo, p);
    }

    // the site with lexicographic index lex (any parity); *parity gets its parity
    __device__ __forceinline__ static EoSite from_lex(const LatDesc& d, uint32_t lex, int* parity)
    {
        const uint32_t r = fdiv(lex, d.div_ns);
        const uint32_t x = lex - r * (uint32_t)d.Ns;
        const uint32_t q = fdiv(r, d.div_ns);
        const uint32_t y = r - q * (uint32_t)d.Ns;
        const uint32_t t = fdiv(q, d.div_ns);
        const uint32_t z = q - t * (uint32_t)d.Ns;
        const int p = (int)((x + y + z + t) & 1u);
        *parity = p;
        return EoSite(d, lex >> 1, p);
    }

    // eo offsets of x + e_d (plus) and x - e_d (minus), wrap included
    __device__ __forceinline__ void hops(int* plus, int* minus) const
    {
        const int b = c[0] & 1;
        const int nh = (int)Nh;
        plus[0] = b ? (c[0] == Ns - 1 ? 1 - nh : 1) : 0;
        minus[0] = b ? 0 : (c[0] == 0 ? nh - 1 : -1);
        int st = nh;
#pragma unroll
        for (int d = 1; d < 4; ++d) {
            const int L = d == 3 ? Nt : Ns;
            plus[d] = c[d] == L - 1 ? -(L - 1) * st : st;
            minus[d] = c[d] == 0 ? (L - 1) * st : -st;
            st *= Ns;
        }
    }

    __device__ __forceinline__ uint32_t lex() const { return (uint32_t)c[0] + (uint32_t)Ns * r; }

    __device__ __forceinline__ int extent(int d) const { return d == 3 ? Nt : Ns; }

    // row stride of direction d (d >= 1)
    __device__ __forceinline__ uint32_t rstride(int d) const
    {
        return d == 1 ? 1u : (d == 2 ? (uint32_t)Ns : (uint32_t)Ns * (uint32_t)Ns);
    }

    // even/odd index of x + s1 e_d1 + s2 e_d2 (s = -1, 0, +1; d1 != d2)
    __device__ __forceinline__ uint32_t nb(int d1, int s1, int d2 = 0, int s2 = 0) const
    {
        int x = c[0];
        int rr = (int)r;
        auto step = [&](int d, int s) {
            if (s == 0) return;
            const int L = extent(d);
            int v = c[d] + s;
            int delta = s;
            if (v == L) delta = s - L;
            else if (v < 0) delta = s + L;
            if (d == 0) x += delta;
            else rr += delta * (int)rstride(d);
        };
        step(d1, s1);
        step(d2, s2);
        return (uint32_t)(x >> 1) + Nh * (uint32_t)rr;
    }
};

}  // namespace su2
