// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sidp {

constexpr int kMaxP = 7;
constexpr int kMaxN = kMaxP + 1;

enum Law { LAW_BURGERS = 1, LAW_EULER = 2, LAW_ADVECTION = 3 };

// Physical parameters of a law.
struct LawParams {
  double gamma;      // Euler
  double beta[2];    // advection
};

// Reference-element tables for one degree p, in the stage precision T.
template <typename T>
struct Tables {
  T w[kMaxN];             // Gauss-Lobatto weights on [0,1]
  T D[kMaxN * kMaxN];     // (D_1D)_{ij} = w_i phi_j'(xi_i), row-major
};

// Per-stage statistics, reduced with atomics (non-negative floats stored as bit patterns).
struct StageStats {
  unsigned long long max_bound_violation;   // double bits
  unsigned long long max_entropy_violation; // double bits
  unsigned int rootfind_max_iters;
  unsigned int pad;
  unsigned long long rootfind_cap_hits;
};

// One problem instance as seen by the kernels.
template <typename T>
struct Instance {
  const T* uin;      // stage input state, [nc][N]
  const T* u0;       // u^n (RK combination), [nc][N]
  T* uout;           // stage output, [nc][N]
  const T* ghost[4]; // exact-state ghost traces [nc][n_side*(p+1)] (or null)
  const double* dt;  // device scalar
  long long N;       // nodes per field
  int nx, ny;
  int bc[4];
  double h;
  T c0, c1;          // RK combination uout = c0 u0 + c1 FE(uin)
  // debug outputs (null = off), per node
  double* dbg_lo;
  double* dbg_hi;
  double* dbg_K;
  double* dbg_alpha;
  StageStats* stats; // null = off
};

template <typename T>
struct StageLaunch {
  Instance<T> inst;
  Tables<T> tab;
  LawParams lp;
  int limiter;
};

// Launchers (one translation unit per law and precision).
template <typename T> cudaError_t launch_stage(int law, int p, const StageLaunch<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_dt(int law, int p, const StageLaunch<T>& a,
                                            unsigned long long* dtmin_bits, cudaStream_t s);

// Host tables (float64), computed once.
void gll_tables(int p, double* xi, double* w, double* D);

}  // namespace sidp

namespace sidp {
// Per-law launchers, explicitly specialised in inst_<law>_<precision>.cu.
template <int LAW, typename T> cudaError_t launch_stage_law(int p, const StageLaunch<T>& a, cudaStream_t s);
template <int LAW, typename T>
cudaError_t launch_dt_law(int p, const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s);
#define SIDP_DECLARE(LAWID, TT)                                                                      \
  template <> cudaError_t launch_stage_law<LAWID, TT>(int, const StageLaunch<TT>&, cudaStream_t);   \
  template <> cudaError_t launch_dt_law<LAWID, TT>(int, const StageLaunch<TT>&, unsigned long long*, \
                                                   cudaStream_t);
SIDP_DECLARE(LAW_BURGERS, double)
SIDP_DECLARE(LAW_BURGERS, float)
SIDP_DECLARE(LAW_EULER, double)
SIDP_DECLARE(LAW_EULER, float)
SIDP_DECLARE(LAW_ADVECTION, double)
SIDP_DECLARE(LAW_ADVECTION, float)
#undef SIDP_DECLARE
}  // namespace sidp
