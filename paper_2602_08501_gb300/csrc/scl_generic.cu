// Stage-1 SC-list kernels for an arbitrary frozen set, checked at run time.
// One segment width (32 lanes = one frame per warp) serves every list size.
#include "scl_impl.cuh"

namespace mpwsd {
using namespace scl_detail;

cudaError_t launch_scl_generic(const CodeDev &c, const SclArgs &a, cudaStream_t s) {
    FrozenRT fz{c.frozen_lo, c.frozen_hi};
    if (c.n == 32) return launch_one<32, 32>(c, a, fz, s);
    if (c.n == 64) return launch_one<64, 32>(c, a, fz, s);
    return launch_one<128, 32>(c, a, fz, s);
}

}  // namespace mpwsd
