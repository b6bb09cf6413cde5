// heatbath_f64_small.cu -- FP64 phase-kernel instantiations with 64 and 32
// threads per block (tiny lattices over many SMs).
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f64_small(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s)
{
    switch (cfg) {
    case 4: return launch_phase_shape<double, LAUNCH_CFG[1][4].threads, LAUNCH_CFG[1][4].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 5: return launch_phase_shape<double, LAUNCH_CFG[1][5].threads, LAUNCH_CFG[1][5].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 6: return launch_phase_shape<double, LAUNCH_CFG[1][6].threads, LAUNCH_CFG[1][6].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 7: return launch_phase_shape<double, LAUNCH_CFG[1][7].threads, LAUNCH_CFG[1][7].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace su2
