// Persistent step kernel (md_step.cuh), mixed instantiations for 16 and 32 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(m, MD_PREC_MIXED, 16)
MD_STEP_DEFINE(m, MD_PREC_MIXED, 32)

}  // namespace mdk
