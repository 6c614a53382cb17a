// Stage-1 dispatch: Reed-Muller frozen sets use kernels compiled with a
// constant frozen mask; any other frozen set uses the run-time-checked kernel.
#include "scl_impl.cuh"

namespace mpwsd {

cudaError_t launch_scl_rm15(const CodeDev &c, const SclArgs &a, cudaStream_t s);
cudaError_t launch_scl_rm26(const CodeDev &c, const SclArgs &a, cudaStream_t s);
cudaError_t launch_scl_rm27(const CodeDev &c, const SclArgs &a, cudaStream_t s);
cudaError_t launch_scl_generic(const CodeDev &c, const SclArgs &a, cudaStream_t s);

int rm_specialisation(int n, uint64_t lo, uint64_t hi) {
    if (n == 32 && lo == (rm_mask(5, 1, 0) & 0xffffffffull)) return 1;
    if (n == 64 && lo == rm_mask(6, 2, 0)) return 2;
    if (n == 128 && lo == rm_mask(7, 2, 0) && hi == rm_mask(7, 2, 1)) return 3;
    return 0;
}

cudaError_t launch_scl(const CodeDev &c, const SclArgs &a, cudaStream_t s) {
    switch (c.rm_spec) {
        case 1: return launch_scl_rm15(c, a, s);
        case 2: return launch_scl_rm26(c, a, s);
        case 3: return launch_scl_rm27(c, a, s);
        default: return launch_scl_generic(c, a, s);
    }
}

}  // namespace mpwsd
