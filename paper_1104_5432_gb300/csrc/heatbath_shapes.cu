// heatbath_shapes.cu -- phase-kernel instantiations for two launch shapes
// of one row of the shape table.  The build compiles this file once per
// pair, with SU2_ROW = 0 (FP32), 1 (FP64) or 2 (FP32 site pairs) and
// SU2_FIRST the first shape index of the pair, so that the shapes compile
// in parallel.
#include <type_traits>

#include "heatbath_kernel.cuh"

#if !defined(SU2_ROW) || !defined(SU2_FIRST)
#error "compile with -DSU2_ROW=<0|1|2> -DSU2_FIRST=<even shape index>"
#endif

namespace su2 {

template <int ROW, int FIRST>
cudaError_t launch_phase_pair(const Ctx& c, int cfg, int mu, int parity, bool plaq, int32_t* dbg,
                              bool hyb, cudaStream_t s)
{
    using T = typename std::conditional<ROW == ROW_F64, double, float>::type;
    constexpr bool PAIRS = ROW == ROW_F32_PAIRS;
    constexpr LaunchCfg A = LAUNCH_CFG[ROW][FIRST];
    constexpr LaunchCfg B = LAUNCH_CFG[ROW][FIRST + 1];
    if (cfg == FIRST)
        return launch_phase_shape<T, A.threads, A.min_blocks, A.slab, A.rounds, A.persistent,
                                  PAIRS, A.group, A.stage>(c, mu, parity, plaq, dbg, hyb, s);
    if (cfg == FIRST + 1)
        return launch_phase_shape<T, B.threads, B.min_blocks, B.slab, B.rounds, B.persistent,
                                  PAIRS, B.group, B.stage>(c, mu, parity, plaq, dbg, hyb, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_phase_pair<SU2_ROW, SU2_FIRST>(const Ctx&, int, int, int, bool, int32_t*,
                                                           bool, cudaStream_t);

}  // namespace su2
