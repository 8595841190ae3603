// Persistent step kernel (md_step.cuh), double-float instantiations for 16 and 32 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(e, MD_PREC_DF, 16)
MD_STEP_DEFINE(e, MD_PREC_DF, 32)

}  // namespace mdk
