// Persistent step kernel, mixed precision instantiations (see md_step.cuh).
#include "md_step.cuh"

namespace mdk {

cudaError_t launch_step32(const Atoms &A, const Cells &C, const Pot &P, int lanes, const StepParams &sp,
                          GridBarrier *bar, unsigned long long *stamps, int *grid_out, cudaStream_t s) {
    return st::launch_prec<MD_PREC_MIXED>(A, C, P, lanes, sp, bar, stamps, grid_out, s);
}

}  // namespace mdk
