// Persistent step kernel (md_step.cuh), double-float instantiations for 1 and 2 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(e, MD_PREC_DF, 1)
MD_STEP_DEFINE(e, MD_PREC_DF, 2)

}  // namespace mdk
