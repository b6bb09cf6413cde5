// cluster.cu -- one heat-bath sweep of a small FP32 lattice in one launch,
// the whole lattice held in the distributed shared memory of one
// thread-block cluster.
//
// A small lattice (8^4: 2048 link updates per phase) spends most of a sweep
// in launch gaps and in the dependent chain of one update, not in memory
// traffic.  Here the CTAs of one cluster (up to 16 SMs) copy the lattice's
// links from global memory into their shared memory, run the eight
// checkerboard phases with the hardware cluster barrier between them (no
// global-memory flag, no spin), finish the sweep (the fused plaquette in a
// fixed order, the sweep counter) and copy the links back: one launch per
// sweep instead of nine.  Every link is updated by update_link, the body of
// the one-link-per-thread kernel, on the same random streams, so the links
// are bit-identical to every other FP32 launch shape.
//
// Layout: CTA r of a cluster of S holds, for each (mu, parity), the links
// eo in [r C, (r + 1) C), C = Vh / S, as float4s at shared-memory offset
// (mu 2 + parity) C + (eo - r C).  A neighbour link of another CTA is read
// with mapa + ld.shared::cluster; a CTA writes only its own links.
#include "heatbath_kernel.cuh"

namespace su2 {

// the links of the cluster, read where they live; written by their owner
struct ClusterLinks {
    uint32_t base;  // shared-window address of this CTA's links
    uint32_t C;     // links per (mu, parity) per CTA
    FastDiv div_c;
    LinkCheck chk;  // bounds-checked builds: a bad index is recorded, link 0 read
    __device__ __forceinline__ Quat<float> load(int mu, int p, uint32_t eo) const
    {
        if (!chk.ok(mu, p, eo)) eo = 0;
        const uint32_t r = fdiv(eo, div_c);
        const uint32_t a = base + (((uint32_t)(mu * 2 + p) * C + (eo - r * C)) << 4);
        uint32_t ra;
        asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
        float4 v;
        // volatile: never moved across the cluster barriers
        asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(ra));
        return {v.x, v.y, v.z, v.w};
    }
};

// all threads of all CTAs of the cluster; the release/acquire pair orders
// every shared-memory write before it with every read after it
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// One phase (MU, p) on this CTA's links: thread t updates eo = r C + t,
// r C + t + NT, ...; the plaquette part of the staple (PLAQ) goes into the
// warp's FP64 partial, lane 0.
template <int MU, bool PLAQ, bool HYB, int NT>
__device__ __forceinline__ void cluster_phase(const LatDesc& D, const ClusterLinks& CU, float4* own,
                                              uint32_t rank, int p, uint64_t sw, double& wplaq,
                                              uint32_t& ntrial, uint32_t& ncap)
{
    const uint32_t C = CU.C;
    float plaq = 0.0f;
    for (uint32_t o = threadIdx.x; o < C; o += NT) {
        const uint32_t i = rank * C + o;
        const EoSite s(D, i, p);
        Quat<float> un, P;
        const int32_t tr = update_link<float, MU, PLAQ, HYB>(CU, D, s, i, p, sw, &un, &P);
        float4& slot = own[(uint32_t)(MU * 2 + p) * C + o];
        if (tr >= 0) {
            slot = make_float4(un.a0, un.a1, un.a2, un.a3);
        } else {
            ++ncap;
            if (PLAQ) un = {slot.x, slot.y, slot.z, slot.w};
        }
        ntrial += tr > 0 ? (uint32_t)tr : (tr < 0 ? (uint32_t)KP_CAP : 0u);
        if (PLAQ) plaq = add_(plaq, qretr(un, P));
    }
    if (PLAQ) {
        const float wp = warp_sum_t(plaq);
        if ((threadIdx.x & 31) == 0) wplaq += (double)wp;
    }
}

template <int MU, bool HYB, int NT>
__device__ __forceinline__ void cluster_mu(const LatDesc& D, const ClusterLinks& CU, float4* own,
                                           uint32_t rank, uint64_t sw, bool pl, double& wplaq,
                                           uint32_t& ntrial, uint32_t& ncap)
{
    cluster_phase<MU, false, HYB, NT>(D, CU, own, rank, 0, sw, wplaq, ntrial, ncap);
    cluster_sync();
    if (MU >= 1 && pl)
        cluster_phase<MU, (MU >= 1), HYB, NT>(D, CU, own, rank, 1, sw, wplaq, ntrial, ncap);
    else
        cluster_phase<MU, false, HYB, NT>(D, CU, own, rank, 1, sw, wplaq, ntrial, ncap);
    cluster_sync();
}

// One sweep of lattice 0 of a single-lattice handle.  Grid: one cluster of
// S CTAs of NT threads, 8 C float4s of dynamic shared memory per CTA.
template <bool HYB, int NT>
__global__ void __launch_bounds__(NT, 1)
hb_cluster_kernel(Ctx ctx, uint32_t C, FastDiv div_c, int pl)
{
    extern __shared__ float4 own[];
    __shared__ double wsum[NT / 32];
    __shared__ double cta_part[CLUSTER_MAX];
    LatDesc* const Dw = ctx.desc;
    // a register copy: the barriers' memory clobbers would otherwise reload
    // the geometry and the coupling from global memory in every phase
    const LatDesc D = *Dw;
    const uint32_t rank = cluster_rank();
    const uint32_t S = gridDim.x;
    const uint32_t Vh = D.Vh;
    const uint64_t sw = D.sweep;
    float4* const glob = reinterpret_cast<float4*>(static_cast<char*>(ctx.links) + D.link_off);

    for (uint32_t k = threadIdx.x; k < 8 * C; k += NT) {
        const uint32_t mp = k / C;
        own[k] = glob[(size_t)mp * Vh + rank * C + (k - mp * C)];
    }
    cluster_sync();  // every CTA's links are in place

    ClusterLinks CU{(uint32_t)__cvta_generic_to_shared(own), C, div_c, {}};
#ifdef SU2_CHECK_BOUNDS
    CU.chk = {ctx.status, Vh};
#endif
    double wplaq = 0.0;
    uint32_t ntrial = 0, ncap = 0;
    const bool plq = pl != 0;
    cluster_mu<0, HYB, NT>(D, CU, own, rank, sw, plq, wplaq, ntrial, ncap);
    cluster_mu<1, HYB, NT>(D, CU, own, rank, sw, plq, wplaq, ntrial, ncap);
    cluster_mu<2, HYB, NT>(D, CU, own, rank, sw, plq, wplaq, ntrial, ncap);
    cluster_mu<3, HYB, NT>(D, CU, own, rank, sw, plq, wplaq, ntrial, ncap);

    // links back to global memory (own links only: no remote reads left)
    for (uint32_t k = threadIdx.x; k < 8 * C; k += NT) {
        const uint32_t mp = k / C;
        glob[(size_t)mp * Vh + rank * C + (k - mp * C)] = own[k];
    }
    // trial counts and cap hits, as the phase kernels count them
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wt = __reduce_add_sync(0xffffffffu, ntrial);
    const uint32_t wc = __reduce_add_sync(0xffffffffu, ncap);
    if (lane == 0) {
        const uint32_t gw = rank * (NT / 32) + w;
        atomicAdd(ctx.trial_slots + (gw % TRIAL_SLOTS), (unsigned long long)wt);
        if (wc) {
            atomicAdd(&Dw->caps, (unsigned long long)wc);
            atomicOr(ctx.status, STATUS_CAP_HIT);
        }
    }
    // the fused plaquette: warps in order, then CTAs in order on CTA 0
    if (plq) {
        if (lane == 0) wsum[w] = wplaq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < NT / 32; ++k) t += wsum[k];
            const uint32_t a = (uint32_t)__cvta_generic_to_shared(&cta_part[rank]);
            uint32_t ra;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(0u));
            asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(t) : "memory");
        }
    }
    cluster_sync();  // the CTAs' sums are on CTA 0; nobody reads remote memory after this
    if (rank == 0 && threadIdx.x == 0) {
        atomicAdd(&Dw->updates, 8ull * (unsigned long long)Vh);
        if (plq) {
            double tot = 0.0;
            for (uint32_t r = 0; r < S; ++r) tot += cta_part[r];
            const double P = tot / (6.0 * (double)D.V);
            const uint64_t k = sw - D.sweep_base;
            ctx.ring[k % PLAQ_RING] = P;
            if (D.plaq_out) D.plaq_out[k] = P;
        }
        Dw->sweep = sw + 1;
    }
}

// cluster size and shared memory for lattice 0, or false when the lattice
// does not fit: the largest S in {16, 8, 4, 2} dividing Vh whose share of
// the links fits a CTA
bool cluster_geometry(uint32_t Vh, int dtype_f32, int n, ClusterGeom* g)
{
    if (!dtype_f32 || n != 1) return false;
    int max_smem = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return false;
    // static shared memory of the kernel: warp and CTA partials
    const size_t room = (size_t)max_smem - 8 * (1024 / 32) - 8 * CLUSTER_MAX;
    for (int S = CLUSTER_MAX; S >= 2; S /= 2) {
        if (Vh % (uint32_t)S) continue;
        const uint32_t C = Vh / (uint32_t)S;
        if ((size_t)8 * C * sizeof(float4) > room) continue;
        g->S = S;
        g->C = C;
        g->div_c = make_fastdiv(C);
        g->threads = C <= 128 ? 128 : 1024;
        g->smem = (size_t)8 * C * sizeof(float4);
        return true;
    }
    return false;
}

template <bool HYB, int NT>
static cudaError_t launch_cluster_nt(const Ctx& c, const ClusterGeom& g, bool plaq, cudaStream_t s)
{
    auto k = hb_cluster_kernel<HYB, NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.S);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)g.S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, c, g.C, g.div_c, plaq ? 1 : 0);
}

cudaError_t launch_cluster_sweep(const Ctx& c, const ClusterGeom& g, bool plaq, bool hyb,
                                 cudaStream_t s)
{
    if (g.threads == 128)
        return hyb ? launch_cluster_nt<true, 128>(c, g, plaq, s)
                   : launch_cluster_nt<false, 128>(c, g, plaq, s);
    return hyb ? launch_cluster_nt<true, 1024>(c, g, plaq, s)
               : launch_cluster_nt<false, 1024>(c, g, plaq, s);
}

// whether one cluster of g.S CTAs with this shared memory can be resident
bool cluster_launchable(const ClusterGeom& g)
{
    auto k = g.threads == 128 ? hb_cluster_kernel<false, 128> : hb_cluster_kernel<false, 1024>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.S);
    cfg.blockDim = dim3((unsigned)g.threads);
    cfg.dynamicSmemBytes = g.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)g.S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

}  // namespace su2
