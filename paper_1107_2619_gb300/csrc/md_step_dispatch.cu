// Persistent step kernel: the precision and lane-count dispatch (the instantiations live in
// md_step_{m,d}_{a,b,c}.cu).
#include "md_step.cuh"

namespace mdk {

cudaError_t launch_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                        const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, int *grid_out,
                        cudaStream_t s) {
    const bool fp64 = precision == MD_PREC_FP64;
    switch (lanes) {
        case 1: return fp64 ? MD_STEP_FN(d, 1)(A, C, P, sp, bar, stamps, grid_out, s)
                            : MD_STEP_FN(m, 1)(A, C, P, sp, bar, stamps, grid_out, s);
        case 2: return fp64 ? MD_STEP_FN(d, 2)(A, C, P, sp, bar, stamps, grid_out, s)
                            : MD_STEP_FN(m, 2)(A, C, P, sp, bar, stamps, grid_out, s);
        case 4: return fp64 ? MD_STEP_FN(d, 4)(A, C, P, sp, bar, stamps, grid_out, s)
                            : MD_STEP_FN(m, 4)(A, C, P, sp, bar, stamps, grid_out, s);
        case 8: return fp64 ? MD_STEP_FN(d, 8)(A, C, P, sp, bar, stamps, grid_out, s)
                            : MD_STEP_FN(m, 8)(A, C, P, sp, bar, stamps, grid_out, s);
        case 16: return fp64 ? MD_STEP_FN(d, 16)(A, C, P, sp, bar, stamps, grid_out, s)
                             : MD_STEP_FN(m, 16)(A, C, P, sp, bar, stamps, grid_out, s);
        case 32: return fp64 ? MD_STEP_FN(d, 32)(A, C, P, sp, bar, stamps, grid_out, s)
                             : MD_STEP_FN(m, 32)(A, C, P, sp, bar, stamps, grid_out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mdk
