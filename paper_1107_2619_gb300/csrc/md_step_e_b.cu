// Persistent step kernel (md_step.cuh), double-float instantiations for 4 and 8 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(e, MD_PREC_DF, 4)
MD_STEP_DEFINE(e, MD_PREC_DF, 8)

}  // namespace mdk
