// heatbath_f64.cu -- FP64 phase-kernel instantiations, 128 and 256
// threads per block; the small-block shapes are in heatbath_f64_small.cu.
#include "heatbath_kernel.cuh"

namespace su2 {

cudaError_t launch_phase_f64_small(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s);

cudaError_t launch_phase_f64(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                             bool hyb, cudaStream_t s)
{
    if (LAUNCH_CFG[1][cfg & 7].threads < 128)
        return launch_phase_f64_small(c, cfg, mu, parity, plaq, dbg, hyb, s);
    switch (cfg) {
    case 0: return launch_phase_shape<double, LAUNCH_CFG[1][0].threads, LAUNCH_CFG[1][0].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 1: return launch_phase_shape<double, LAUNCH_CFG[1][1].threads, LAUNCH_CFG[1][1].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 2: return launch_phase_shape<double, LAUNCH_CFG[1][2].threads, LAUNCH_CFG[1][2].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    case 3: return launch_phase_shape<double, LAUNCH_CFG[1][3].threads, LAUNCH_CFG[1][3].min_blocks, false>(c, mu, parity, plaq, dbg, hyb, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace su2
