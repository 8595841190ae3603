// Persistent step kernel (md_step.cuh), mixed instantiations for 1 and 2 lanes per atom.
#include "md_step.cuh"

namespace mdk {

MD_STEP_DEFINE(m, MD_PREC_MIXED, 1)
MD_STEP_DEFINE(m, MD_PREC_MIXED, 2)

}  // namespace mdk
