// Persistent step kernel (md_step.cuh), FP64 instantiations for 1 and 2 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(d, MD_PREC_FP64, 1)
MD_STEP_DEFINE(d, MD_PREC_FP64, 2)

}  // namespace mdk
