// Time-step reduction that allocates nothing (sidp_compute_dt_static).
//
// Who needs it: callers that cannot allocate device memory at the point where they need a time
// step -- e.g. a host application that hands all device memory to its own pool allocator and
// forbids other allocations, a real-time loop in which cudaMalloc's implicit synchronisation and
// unbounded latency are not acceptable, or a caller that only holds a device pointer to a state
// it owns and no libsidp context.  sidp_compute_dt allocates through its context; this entry
// point takes the state and the output as caller-owned device pointers and keeps its scratch in
// a fixed file-scope device array instead.
//
// Scratch: g_dt_partials, one float64 partial minimum per thread block, kMaxStaticBlocks of them
// (512 KiB, held by every GPU that loads the library until the process exits).  That bounds the
// problem size to kMaxStaticBlocks * 256 nodes; larger states are rejected with SIDP_ERR_ARG.
// Every slot a call reads is written by the same call first, so nothing needs clearing between
// calls, but all calls share the one array: calls whose kernels overlap on the GPU (two streams,
// or two host threads) race and may return each other's result.  Serialise them.
//
// Set-up: the device address of g_dt_partials is looked up with cudaGetSymbolAddress the first
// time the entry point runs on a device (with that device current) and cached per device.  Make
// that first call outside any stream capture.  The cached address belongs to the device's primary
// context: resetting the device (cudaDeviceReset) after the first call is not supported.
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "sidp.h"
#include "sidp_laws.cuh"
#include "sidp_internal.h"

namespace sidp {
namespace {

constexpr int kStaticThreads = 256;
constexpr long long kMaxStaticBlocks = 65536;

__device__ __align__(256) double g_dt_partials[kMaxStaticBlocks];

// Same neighbour rule as the stage kernel: periodic wraps, outflow copies the node itself.
template <int P, int NC, typename T>
__device__ __forceinline__ void static_neighbor(const T* u, long long N, int nx, int ny, const int* bc, int side,
                                                long long e, int ex, int ey, int pos, const T* own, T* out) {
  constexpr int n = P + 1, NN = n * n;
  long long ne = -1;
  int nd = 0;
  switch (side) {
    case 0: nd = pos * n + P; ne = (ex > 0) ? e - 1 : (bc[0] == 0 ? e + (nx - 1) : -1); break;
    case 1: nd = pos * n; ne = (ex < nx - 1) ? e + 1 : (bc[1] == 0 ? e - (nx - 1) : -1); break;
    case 2: nd = P * n + pos; ne = (ey > 0) ? e - nx : (bc[2] == 0 ? e + (long long)(ny - 1) * nx : -1); break;
    default: nd = pos; ne = (ey < ny - 1) ? e + nx : (bc[3] == 0 ? e - (long long)(ny - 1) * nx : -1); break;
  }
#pragma unroll
  for (int f = 0; f < NC; ++f) out[f] = (ne >= 0) ? u[f * N + ne * NN + nd] : own[f];
}

// One partial minimum of m_i / (2 sum_{j != i} d-hat_ij) (Eq. cfl-low) per block.
template <int P, class LAW, typename T>
__global__ void __launch_bounds__(kStaticThreads)
k_dt_static(const T* __restrict__ u, long long N, int nx, int ny, int4 bc4, double h, Tables<T> tab,
            LawParamsT<T> lp, double* partials) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  using Aux = typename LAW::Aux;
  const int bc[4] = {bc4.x, bc4.y, bc4.z, bc4.w};
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double val = DBL_MAX;
  if (g < N) {
    const long long e = g / NN;
    const int node = (int)(g - e * NN), a = node / n, b = node - a * n;
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    T uu[NC], v[NC];
    Aux ax, av;
#pragma unroll
    for (int f = 0; f < NC; ++f) uu[f] = u[f * N + g];
    LAW::aux(uu, ax, lp);
    T lam[4];
#pragma unroll
    for (int side = 0; side < 4; ++side) {
      const int k = side >> 1;
      const bool lower = (side & 1) == 0;
      const int idx = (k == 0) ? b : a;
      if (lower ? (idx > 0) : (idx < P)) {
        const long long gn = g + (k == 0 ? (lower ? -1 : 1) : (lower ? -n : n));
#pragma unroll
        for (int f = 0; f < NC; ++f) v[f] = u[f * N + gn];
      } else {
        static_neighbor<P, NC>(u, N, nx, ny, bc, side, e, ex, ey, (k == 0) ? a : b, uu, v);
      }
      LAW::aux(v, av, lp);
      lam[side] = lower ? LAW::lam(k, v, av, uu, ax, lp) : LAW::lam(k, uu, ax, v, av, lp);
    }
    // per-node bound in the stage precision, like the context's time-step kernel
    const T hT = T(h), wa = tab.w[a], wb = tab.w[b];
    const T sumd = T(0.5) * hT * wa * (lam[0] + lam[1]) + T(0.5) * hT * wb * (lam[2] + lam[3]);
    if (sumd > T(0)) val = (double)fdiv(hT * hT * wa * wb, T(2) * sumd);  // the context kernel's division
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, o));
  __shared__ double red[kStaticThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int i = 1; i < kStaticThreads / 32; ++i) m = fmin(m, red[i]);
    partials[blockIdx.x] = m;
  }
}

// min over the partials (fixed order), times the CFL number; 0 when no wave moves.
__global__ void k_dt_static_final(const double* partials, long long nblocks, double cfl, double* dt_out) {
  __shared__ double red[kStaticThreads];
  double m = DBL_MAX;
  for (long long i = threadIdx.x; i < nblocks; i += blockDim.x) m = fmin(m, partials[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *dt_out = (red[0] < DBL_MAX) ? cfl * red[0] : 0.0;
}

template <int P, class LAW, typename T>
cudaError_t launch_static(const sidp_config* cfg, const void* d_state, long long N, double h, double* partials,
                          double* d_dt, cudaStream_t s) {
  Tables<T> tab{};
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  gll_tables(P, xi, w, D);
  for (int i = 0; i <= P; ++i) tab.w[i] = T(w[i]);
  const LawParamsT<T> lp = make_law_params<T>(cfg->gamma, cfg->adv_beta);
  const long long blocks = (N + kStaticThreads - 1) / kStaticThreads;
  const int4 bc4 = make_int4(cfg->bc[0], cfg->bc[1], cfg->bc[2], cfg->bc[3]);
  k_dt_static<P, LAW, T><<<(unsigned)blocks, kStaticThreads, 0, s>>>(static_cast<const T*>(d_state), N, cfg->nx,
                                                                       cfg->ny, bc4, h, tab, lp, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dt_static_final<<<1, kStaticThreads, 0, s>>>(partials, blocks, cfg->cfl, d_dt);
  return cudaGetLastError();
}

template <class LAW, typename T>
cudaError_t dispatch_static(const sidp_config* cfg, const void* d_state, long long N, double h, double* partials,
                            double* d_dt, cudaStream_t s) {
  switch (cfg->p) {
    case 1: return launch_static<1, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 2: return launch_static<2, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 3: return launch_static<3, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 4: return launch_static<4, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 5: return launch_static<5, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 6: return launch_static<6, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    case 7: return launch_static<7, LAW, T>(cfg, d_state, N, h, partials, d_dt, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t dispatch_static_law(const sidp_config* cfg, const void* d_state, long long N, double h,
                                double* partials, double* d_dt, cudaStream_t s) {
  switch (cfg->law) {
    case LAW_BURGERS: return dispatch_static<LawBurgers<T>, T>(cfg, d_state, N, h, partials, d_dt, s);
    case LAW_EULER: return dispatch_static<LawEuler<T>, T>(cfg, d_state, N, h, partials, d_dt, s);
    case LAW_ADVECTION: return dispatch_static<LawAdvection<T>, T>(cfg, d_state, N, h, partials, d_dt, s);
    default: return cudaErrorInvalidValue;
  }
}

std::mutex g_static_mu;
double* g_static_ptr[64] = {nullptr};

}  // namespace
}  // namespace sidp

extern "C" sidp_status sidp_compute_dt_static(const sidp_config* cfg, const void* d_state, double* d_dt,
                                              void* cuda_stream) {
  using namespace sidp;
  std::string msg;
  const sidp_status st = validate_config(cfg, msg);  // the context's checks (gamma, periodic pairing, ...)
  if (st != SIDP_OK) { set_last_error(msg); return st; }
  if (!d_state || !d_dt) { set_last_error("null device pointer"); return SIDP_ERR_ARG; }
  if (cfg->law == SIDP_LAW_ADVECTION_VAR2D) { set_last_error("variable-velocity advection is not supported here"); return SIDP_ERR_ARG; }
  if (cfg->unsparsified) {  // the dense operator's bound (every in-element pair) is smaller: not computed here
    set_last_error("the unsparsified mode is not supported here");
    return SIDP_ERR_ARG;
  }
  for (int s = 0; s < 4; ++s)
    if (cfg->bc[s] != SIDP_BC_PERIODIC && cfg->bc[s] != SIDP_BC_OUTFLOW) {  // no ghost traces here
      set_last_error("periodic and outflow sides only");
      return SIDP_ERR_ARG;
    }
  const double h = (cfg->x1 - cfg->x0) / cfg->nx;
  const long long N = (long long)cfg->nx * cfg->ny * (cfg->p + 1) * (cfg->p + 1);
  if ((N + kStaticThreads - 1) / kStaticThreads > kMaxStaticBlocks) {  // beyond the scratch
    set_last_error("state larger than the fixed scratch allows (16,777,216 nodes)");
    return SIDP_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SIDP_ERR_CUDA;
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_dt_partials) != cudaSuccess || !p) return SIDP_ERR_CUDA;
      g_static_ptr[dev] = static_cast<double*>(p);
    }
    partials = g_static_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const cudaError_t e = (cfg->precision == SIDP_MIXED)
                            ? dispatch_static_law<float>(cfg, d_state, N, h, partials, d_dt, s)
                            : dispatch_static_law<double>(cfg, d_state, N, h, partials, d_dt, s);
  return e == cudaSuccess ? SIDP_OK : SIDP_ERR_CUDA;
}
