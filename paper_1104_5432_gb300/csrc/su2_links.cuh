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
        const uint32_t r = fdiv(j, d.div_nh);
        const uint32_t xh = j - r * (uint32_t)d.Nh;
        const uint32_t r2 = fdiv(r, d.div_ny);
        const uint32_t yl = r - r2 * (uint32_t)d.Ny;
        const uint32_t r3 = fdiv(r2, d.div_ns);
        const uint32_t z = r2 - r3 * (uint32_t)d.Ns;
        const uint32_t ys = fdiv(r3, d.div_nt);
        const uint32_t t = r3 - ys * (uint32_t)d.Nt;
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
