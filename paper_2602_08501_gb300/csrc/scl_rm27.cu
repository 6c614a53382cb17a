// Stage-1 SC-list kernels specialised for the RM(2,7), n = 128 frozen set
// (compile-time frozen checks keep the per-leaf list code to the information leaves).
#include "scl_impl.cuh"

namespace mpwsd {
using namespace scl_detail;

cudaError_t launch_scl_rm27(const CodeDev &c, const SclArgs &a, cudaStream_t s) {
    FrozenCT<rm_mask(7, 2, 0), rm_mask(7, 2, 1)> fz{0, 0};
    return launch_lw<128>(c, a, fz, s);
}

}  // namespace mpwsd
