// Stage and time-step kernels of the euler law in float, degrees 4, 5
// (split into translation units so that the build runs in parallel).
#include "sidp_curved.cuh"
#include "sidp_lines.cuh"
#include "sidp_curved_lines.cuh"

namespace sidp {
SIDP_INSTANTIATE_P(LAW_EULER, LawEuler, float, 4)
SIDP_INSTANTIATE_P(LAW_EULER, LawEuler, float, 5)
}  // namespace sidp
