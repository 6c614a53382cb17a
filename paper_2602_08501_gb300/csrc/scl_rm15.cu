// Stage-1 SC-list kernels specialised for the RM(1,5), n = 32 frozen set
// (compile-time frozen checks keep the per-leaf list code to the information leaves).
#include "scl_impl.cuh"

namespace mpwsd {
using namespace scl_detail;

cudaError_t launch_scl_rm15(const CodeDev &c, const SclArgs &a, cudaStream_t s) {
    FrozenCT<rm_mask(5, 1, 0) & 0xffffffffull, 0> fz{0, 0};
    return launch_lw<32>(c, a, fz, s);
}

}  // namespace mpwsd
