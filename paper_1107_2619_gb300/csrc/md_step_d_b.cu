// Persistent step kernel (md_step.cuh), FP64 instantiations for 4 and 8 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(d, MD_PREC_FP64, 4)
MD_STEP_DEFINE(d, MD_PREC_FP64, 8)

}  // namespace mdk
