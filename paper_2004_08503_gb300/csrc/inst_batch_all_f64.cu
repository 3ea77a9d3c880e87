// Single-launch batch kernels (every degree in one launch) of all laws in double
// (a translation unit of its own so that the build runs in parallel).
#include "sidp_kernels.cuh"

namespace sidp {
template <> cudaError_t launch_batch_all<LAW_BURGERS, double>(const BatchAllLaunch<double>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawBurgers<double>, double>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_EULER, double>(const BatchAllLaunch<double>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawEuler<double>, double>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_ADVECTION, double>(const BatchAllLaunch<double>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawAdvection<double>, double>(b, dt, s);
}
template <> cudaError_t launch_batch_all<LAW_ADVECTION_VAR, double>(const BatchAllLaunch<double>& b, bool dt, cudaStream_t s) {
  return launch_batch_all_law<LawAdvectionVar<double>, double>(b, dt, s);
}
}  // namespace sidp
