// Persistent step kernel (md_step.cuh), FP64 instantiations for 16 and 32 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(d, MD_PREC_FP64, 16)
MD_STEP_DEFINE(d, MD_PREC_FP64, 32)

}  // namespace mdk
