// Persistent step kernel: the precision and lane-count dispatch (the instantiations live in
// md_step_{m,d,e}_{a,b,c}.cu: mixed, FP64, double-float).
#include "md_step.cuh"

namespace mdk {

cudaError_t launch_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                        const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, int *grid_out,
                        cudaStream_t s) {
#define MD_STEP_CASE(T)                                                                  \
    case T:                                                                              \
        if (precision == MD_PREC_FP64) return MD_STEP_FN(d, T)(A, C, P, sp, bar, stamps, grid_out, s); \
        if (precision == MD_PREC_DF) return MD_STEP_FN(e, T)(A, C, P, sp, bar, stamps, grid_out, s);   \
        return MD_STEP_FN(m, T)(A, C, P, sp, bar, stamps, grid_out, s);
    switch (lanes) {
        MD_STEP_CASE(1)
        MD_STEP_CASE(2)
        MD_STEP_CASE(4)
        MD_STEP_CASE(8)
        MD_STEP_CASE(16)
        MD_STEP_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef MD_STEP_CASE
}

// The walk of the step kernel launch_step runs for this context (launch_kind's choice).
int step_walk(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes) {
    if (precision == MD_PREC_FP64 && A.pairs) return kWalkPairs;
    if (precision == MD_PREC_MIXED && lanes <= 8 && P.kind == MD_POT_TABLES && P.ns == 1 &&
        smem_table_bytes(P.kind, P.ns, precision, P.nk) > 0 &&
        (C.tile == kWalkStaged || C.tile == kWalkCells || C.tile == kWalkHalf))
        return C.tile;
    return kWalkList;
}

cudaError_t launch_rebuild_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                                const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, cudaStream_t s) {
    switch (step_walk(A, C, P, precision, lanes)) {
        case kWalkStaged: return st::launch_rebuild_t<kWalkStaged>(A, C, sp, bar, stamps, s);
        case kWalkCells: return st::launch_rebuild_t<kWalkCells>(A, C, sp, bar, stamps, s);
        case kWalkHalf: return st::launch_rebuild_t<kWalkHalf>(A, C, sp, bar, stamps, s);
        case kWalkPairs: return st::launch_rebuild_t<kWalkPairs>(A, C, sp, bar, stamps, s);
        default: return st::launch_rebuild_t<kWalkList>(A, C, sp, bar, stamps, s);
    }
}

}  // namespace mdk
