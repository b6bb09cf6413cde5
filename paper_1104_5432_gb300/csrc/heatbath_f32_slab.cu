// heatbath_f32_slab.cu -- FP32 phase-kernel instantiations that walk the
// lattice in y slabs (the slab entries of LAUNCH_CFG[0]).
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f32_slab(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s)
{
    switch (cfg) {
    case 4: return launch_phase_shape<float, LAUNCH_CFG[0][4].threads, LAUNCH_CFG[0][4].min_blocks, true>(c, mu, parity, plaq, dbg, hyb, s);
    case 5: return launch_phase_shape<float, LAUNCH_CFG[0][5].threads, LAUNCH_CFG[0][5].min_blocks, true>(c, mu, parity, plaq, dbg, hyb, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace su2
