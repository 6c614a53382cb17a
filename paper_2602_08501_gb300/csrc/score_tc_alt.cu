// Tensor-core scoring: the alternative shapes that MPWSD_TUNE_TC_SHAPE selects
// (compiled apart from the defaults so that the library builds in parallel).
#include "score_tc_impl.cuh"

namespace mpwsd {

cudaError_t launch_score_tc_alt(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    if (c.n == 64) {
        switch (c.tc_shape) {
            case 1: return launch_shape<64, 256, 4, 2>(c, a, s);   // four A builders
            case 2: return launch_shape<64, 128, 2, 2>(c, a, s);   // 128-pattern tiles, two accumulators per row block
            case 3: return launch_shape<64, 128, 2, 4>(c, a, s);   // ... with a four-stage tile ring
            default: break;
        }
    } else if (c.n == 128 && c.tc_shape == 1) {
        return launch_shape<128, 128, 4, 2>(c, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mpwsd
