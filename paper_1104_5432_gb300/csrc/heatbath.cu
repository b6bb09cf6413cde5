// heatbath.cu -- sweep orchestration kernels of the SU(2) heat bath: the
// end-of-sweep reduction of the fused plaquette, the per-call parameter
// kernel and the dispatch of the phase kernels (heatbath_kernel.cuh,
// instantiated per pair of launch shapes and precision by
// heatbath_shapes.cu).
#include "su2_internal.h"
#include "su2_reduce.cuh"

namespace su2 {

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
    // partials are per warp: lattice l owns warps [b0, b0 + nb) of each slot
    const uint32_t b0 = ctx.phase_start[l] * ctx.phase_wpb;
    const uint32_t nb = ctx.phase_start[l + 1] * ctx.phase_wpb - b0;
    const uint32_t stride = ctx.phase_blocks * ctx.phase_wpb;
    const uint32_t total = 3 * nb;
    const uint32_t nchunk = (total + SWEEP_CHUNK - 1) / SWEEP_CHUNK;
    if (blockIdx.x >= nchunk) return;

    const uint32_t e0 = blockIdx.x * SWEEP_CHUNK;
    const uint32_t e1 = min(e0 + (uint32_t)SWEEP_CHUNK, total);
    double acc = 0.0;
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += TPB) {
        const uint32_t slot = (e >= nb) + (e >= 2 * nb);
        acc += ctx.plaq_partial[(size_t)slot * stride + b0 + (e - slot * nb)];
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
    D->beta_f = (float)pc.beta[j];
    D->half_inv_beta_f = (float)(0.5 / pc.beta[j]);
    D->half_inv_beta = 0.5 / pc.beta[j];  // inf at beta = 0, where the Haar draw applies
    D->seed = pc.seed[j];
    D->plaq_out = pc.plaq_out[j];
    D->sweep_base = D->sweep;
}

// one pair of launch shapes per instantiation of heatbath_shapes.cu
template <int ROW, int FIRST>
cudaError_t launch_phase_pair(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                              bool hyb, cudaStream_t s);

cudaError_t launch_phase(const Ctx& c, int row, int cfg, int mu, int parity, bool plaq,
                         int32_t* dbg_trials, bool hybrid, cudaStream_t s)
{
    using Fn = cudaError_t (*)(const Ctx&, int, int, int, bool, int32_t*, bool, cudaStream_t);
    static_assert(NUM_LAUNCH_CFG == 14 && NUM_ROWS == 3, "one entry per pair of shapes below");
    static const Fn pairs[NUM_ROWS][NUM_LAUNCH_CFG / 2] = {
        {launch_phase_pair<0, 0>, launch_phase_pair<0, 2>, launch_phase_pair<0, 4>,
         launch_phase_pair<0, 6>, launch_phase_pair<0, 8>, launch_phase_pair<0, 10>,
         launch_phase_pair<0, 12>},
        {launch_phase_pair<1, 0>, launch_phase_pair<1, 2>, launch_phase_pair<1, 4>,
         launch_phase_pair<1, 6>, launch_phase_pair<1, 8>, launch_phase_pair<1, 10>,
         launch_phase_pair<1, 12>},
        {launch_phase_pair<2, 0>, launch_phase_pair<2, 2>, launch_phase_pair<2, 4>,
         launch_phase_pair<2, 6>, launch_phase_pair<2, 8>, launch_phase_pair<2, 10>,
         launch_phase_pair<2, 12>},
    };
    if (row < 0 || row >= NUM_ROWS || cfg < 0 || cfg >= NUM_LAUNCH_CFG) return cudaErrorInvalidValue;
    return pairs[row][cfg >> 1](c, cfg, mu, parity, plaq, dbg_trials, hybrid, s);
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
