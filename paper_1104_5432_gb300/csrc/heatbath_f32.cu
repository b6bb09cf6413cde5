// heatbath_f32.cu -- FP32 phase-kernel instantiations, plain traversal,
// 128..512 threads per block; dispatch to the other FP32 units.
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f32_slab(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s);
cudaError_t launch_phase_f32_small(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s);

cudaError_t launch_phase_f32(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s)
{
    if (LAUNCH_CFG[0][cfg & 7].slab) return launch_phase_f32_slab(c, cfg, mu, parity, plaq, dbg, hyb, s);
    if (LAUNCH_CFG[0][cfg & 7].threads < 128)
        return launch_phase_f32_small(c, cfg, mu, parity, plaq, dbg, hyb, s);
    switch (cfg) {
    case 0: return launch_phase_shape<float, LAUNCH_CFG[0][0].threads, LAUNCH_CFG[0][0].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 1: return launch_phase_shape<float, LAUNCH_CFG[0][1].threads, LAUNCH_CFG[0][1].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 2: return launch_phase_shape<float, LAUNCH_CFG[0][2].threads, LAUNCH_CFG[0][2].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 3: return launch_phase_shape<float, LAUNCH_CFG[0][3].threads, LAUNCH_CFG[0][3].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace su2
