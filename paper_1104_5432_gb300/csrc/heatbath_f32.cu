// heatbath_f32.cu -- FP32 instantiations of the phase kernel for every
// launch shape the autotuner may choose (LAUNCH_CFG[0]).
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f32(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             cudaStream_t s)
{
    switch (cfg) {
    case 0: return launch_phase_shape<float, LAUNCH_CFG[0][0].threads, LAUNCH_CFG[0][0].min_blocks>(c, mu, parity, plaq, dbg, s);
    case 1: return launch_phase_shape<float, LAUNCH_CFG[0][1].threads, LAUNCH_CFG[0][1].min_blocks>(c, mu, parity, plaq, dbg, s);
    case 2: return launch_phase_shape<float, LAUNCH_CFG[0][2].threads, LAUNCH_CFG[0][2].min_blocks>(c, mu, parity, plaq, dbg, s);
    default: return launch_phase_shape<float, LAUNCH_CFG[0][3].threads, LAUNCH_CFG[0][3].min_blocks>(c, mu, parity, plaq, dbg, s);
    }
}

}  // namespace su2
