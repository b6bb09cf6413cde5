// heatbath_f64.cu -- FP64 instantiations of the phase kernel for every
// launch shape the autotuner may choose (LAUNCH_CFG[1]).
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f64(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s)
{
    switch (cfg) {
    case 0: return launch_phase_shape<double, LAUNCH_CFG[1][0].threads, LAUNCH_CFG[1][0].min_blocks, LAUNCH_CFG[1][0].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 1: return launch_phase_shape<double, LAUNCH_CFG[1][1].threads, LAUNCH_CFG[1][1].min_blocks, LAUNCH_CFG[1][1].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 2: return launch_phase_shape<double, LAUNCH_CFG[1][2].threads, LAUNCH_CFG[1][2].min_blocks, LAUNCH_CFG[1][2].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 3: return launch_phase_shape<double, LAUNCH_CFG[1][3].threads, LAUNCH_CFG[1][3].min_blocks, LAUNCH_CFG[1][3].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 4: return launch_phase_shape<double, LAUNCH_CFG[1][4].threads, LAUNCH_CFG[1][4].min_blocks, LAUNCH_CFG[1][4].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 5: return launch_phase_shape<double, LAUNCH_CFG[1][5].threads, LAUNCH_CFG[1][5].min_blocks, LAUNCH_CFG[1][5].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 6: return launch_phase_shape<double, LAUNCH_CFG[1][6].threads, LAUNCH_CFG[1][6].min_blocks, LAUNCH_CFG[1][6].slab>(c, mu, parity, plaq, dbg, hyb, s);
    case 7: return launch_phase_shape<double, LAUNCH_CFG[1][7].threads, LAUNCH_CFG[1][7].min_blocks, LAUNCH_CFG[1][7].slab>(c, mu, parity, plaq, dbg, hyb, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace su2
