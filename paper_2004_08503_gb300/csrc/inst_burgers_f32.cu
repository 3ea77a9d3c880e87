// Stage and time-step kernels of the burgers law in float, degrees 1, 2, 3, 4, 5, 6, 7
// (split into translation units so that the build runs in parallel).
#include "sidp_curved.cuh"
#include "sidp_lines.cuh"
#include "sidp_curved_lines.cuh"

namespace sidp {
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 1)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 2)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 3)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 4)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 5)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 6)
SIDP_INSTANTIATE_P(LAW_BURGERS, LawBurgers, float, 7)
}  // namespace sidp
