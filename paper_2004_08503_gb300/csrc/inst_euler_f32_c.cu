// Stage and time-step kernels of the euler law in float, degrees 6, 7
// (split into translation units so that the build runs in parallel).
#include "sidp_curved.cuh"
#include "sidp_lines.cuh"
#include "sidp_curved_lines.cuh"

namespace sidp {
SIDP_INSTANTIATE_P(LAW_EULER, LawEuler, float, 6)
SIDP_INSTANTIATE_P(LAW_EULER, LawEuler, float, 7)
}  // namespace sidp
