// Persistent step kernel (md_step.cuh), mixed instantiations for 4 and 8 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(m, MD_PREC_MIXED, 4)
MD_STEP_DEFINE(m, MD_PREC_MIXED, 8)

}  // namespace mdk
