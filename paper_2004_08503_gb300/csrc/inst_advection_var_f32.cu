// Stage and time-step kernels of the variable-velocity advection law in float, degrees 1..7
// (split into translation units so that the build runs in parallel).
#include "sidp_curved.cuh"
#include "sidp_lines.cuh"
#include "sidp_curved_lines.cuh"

namespace sidp {
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 1)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 2)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 3)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 4)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 5)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 6)
SIDP_INSTANTIATE_P(LAW_ADVECTION_VAR, LawAdvectionVar, float, 7)
}  // namespace sidp
