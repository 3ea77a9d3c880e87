// Stage and time-step kernels of the burgers law in float (one translation unit per law and
// precision so that the builds run in parallel).
#include "sidp_kernels.cuh"

namespace sidp {
SIDP_INSTANTIATE(LAW_BURGERS, LawBurgers, float)
}  // namespace sidp
