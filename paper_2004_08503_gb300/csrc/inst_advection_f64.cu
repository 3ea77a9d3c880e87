// Stage and time-step kernels of the advection law in double (one translation unit per law and
// precision so that the builds run in parallel).
#include "sidp_kernels.cuh"

namespace sidp {
SIDP_INSTANTIATE(LAW_ADVECTION, LawAdvection, double)
}  // namespace sidp
