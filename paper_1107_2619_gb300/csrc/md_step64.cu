// Persistent step kernel, FP64 instantiations (see md_step.cuh), and the precision dispatch.
#include "md_step.cuh"

namespace mdk {

cudaError_t launch_step32(const Atoms &A, const Cells &C, const Pot &P, int lanes, const StepParams &sp,
                          GridBarrier *bar, unsigned long long *stamps, int *grid_out, cudaStream_t s);

cudaError_t launch_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                        const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, int *grid_out,
                        cudaStream_t s) {
    if (precision == MD_PREC_FP64) return st::launch_prec<MD_PREC_FP64>(A, C, P, lanes, sp, bar, stamps, grid_out, s);
    return launch_step32(A, C, P, lanes, sp, bar, stamps, grid_out, s);
}

}  // namespace mdk
