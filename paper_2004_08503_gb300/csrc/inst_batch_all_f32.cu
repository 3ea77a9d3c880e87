// Single-launch batch kernels (every degree in one launch) of all laws in float
// (a translation unit of its own so that the build runs in parallel).
#include "sidp_kernels.cuh"

namespace sidp {
template <> cudaError_t launch_batch_all<LAW_BURGERS, float>(const BatchAllLaunch<float>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawBurgers<float>, float>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_EULER, float>(const BatchAllLaunch<float>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawEuler<float>, float>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_ADVECTION, float>(const BatchAllLaunch<float>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawAdvection<float>, float>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_ADVECTION_VAR, float>(const BatchAllLaunch<float>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawAdvectionVar<float>, float>(b, dt, s);
}
}  // namespace sidp
