// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cmath>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include "sidp.h"

namespace sidp {

constexpr int kMaxP = 7;
constexpr int kGeoFields = SIDP_GEO_FIELDS;  // per-node metric arrays of a curved mesh
constexpr int GEO_MASS_FIELD = 8;           // index of m_i among them
constexpr int kMaxN = kMaxP + 1;

enum Law { LAW_BURGERS = 1, LAW_EULER = 2, LAW_ADVECTION = 3, LAW_ADVECTION_VAR = 4 };

// Physical parameters of a law.
// Law constants in the stage precision T, computed once on the host (float kernels must not
// convert from float64 per call: float64 throughput on this GPU is a small fraction of float32).
template <typename T>
struct LawParamsT {
  T gamma;      // Euler ratio of specific heats
  T gm1;        // gamma - 1
  T half_gm1;   // (gamma - 1) / 2
  T inv_gm1;    // 1 / (gamma - 1)
  T c_gp;       // (gamma + 1) / (2 gamma)
  T neg_e;      // -(gamma - 1) / (2 gamma)
  T inv_e;      // 2 gamma / (gamma - 1): exponent of the two-rarefaction pressure
  T beta[2];    // advection velocity (variable-velocity law: its constant part)
  T bxy, byx;   // variable-velocity law: beta = (beta[0] + bxy y, beta[1] + byx x)
  int pow7;     // inv_e == 7 (gamma = 1.4): the float path multiplies instead of calling pow
  double gamma_d;  // gamma in float64 (statistics)
};

template <typename T>
inline LawParamsT<T> make_law_params(double gamma, const double* beta, const double* grad = nullptr) {
  LawParamsT<T> p{};
  const double g = gamma > 1.0 ? gamma : 1.4;
  p.gamma = T(g);
  p.gm1 = T(g - 1.0);
  p.half_gm1 = T(0.5 * (g - 1.0));
  p.inv_gm1 = T(1.0 / (g - 1.0));
  p.c_gp = T((g + 1.0) / (2.0 * g));
  p.neg_e = T(-(g - 1.0) / (2.0 * g));
  p.inv_e = T(2.0 * g / (g - 1.0));
  p.beta[0] = T(beta[0]);
  p.beta[1] = T(beta[1]);
  p.bxy = grad ? T(grad[0]) : T(0);
  p.byx = grad ? T(grad[1]) : T(0);
  p.pow7 = (2.0 * g / (g - 1.0) > 7.0 - 1e-12 && 2.0 * g / (g - 1.0) < 7.0 + 1e-12) ? 1 : 0;
  p.gamma_d = g;
  return p;
}

// Element tile shapes (elements along x, y per CTA) for each degree; index 0 is the default (the
// fastest on the Euler float32 path where the candidates were measured) and the autotuner picks
// among them per (law, p, precision).
struct TileShape { int tx, ty; };
constexpr int kNumTiles = 4;
constexpr TileShape kTiles[kMaxP + 1][kNumTiles] = {
    {{0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{8, 8}, {16, 4}, {4, 16}, {16, 8}},  // p=1: 256 / 256 / 256 / 512 threads
    {{4, 7}, {7, 4}, {5, 5}, {7, 7}},     // p=2: 252 / 252 / 225 / 441
    {{4, 4}, {8, 2}, {2, 8}, {8, 4}},     // p=3: 256 / 256 / 256 / 512
    {{2, 5}, {5, 2}, {3, 3}, {4, 5}},     // p=4: 250 / 250 / 225 / 500
    {{7, 1}, {3, 2}, {2, 3}, {3, 4}},     // p=5: 252 / 216 / 216 / 432
    {{1, 5}, {5, 1}, {2, 2}, {3, 3}},     // p=6: 245 / 245 / 196 / 441
    {{1, 4}, {4, 1}, {2, 2}, {4, 2}},     // p=7: 256 / 256 / 256 / 512
};

// Element tiles of the line-parallel stage kernel (one thread per element line; Euler, subcell
// limiting without the smoothness indicator).  Tile index kNumTiles + i selects kLineTiles[p][i].
constexpr int kNumLineTiles = 2;
constexpr TileShape kLineTiles[kMaxP + 1][kNumLineTiles] = {
    {{0, 0}, {0, 0}},
    {{16, 8}, {8, 8}},  // p=1: 256 / 128 threads
    {{8, 8}, {10, 8}},  // p=2: 192 / 240
    {{8, 4}, {8, 8}},   // p=3: 128 / 256
    {{8, 4}, {6, 6}},   // p=4: 160 / 180
    {{4, 4}, {6, 4}},   // p=5: 96 / 144
    {{4, 4}, {4, 2}},   // p=6: 112 / 56
    {{4, 4}, {4, 2}},   // p=7: 128 / 64
};
constexpr int kMaxCand = kNumTiles + kNumLineTiles;
// Batches: the smallest mean instance size (nodes) of a degree group whose tuning includes the line
// kernel's tiles.
constexpr long long kLineMinNodes = 1LL << 21;
// Candidates of the tile autotuner for a law: the node kernel's shapes, then (Euler) the line
// kernel's.
inline int num_tile_candidates(int law) { return kNumTiles + (law == LAW_EULER ? kNumLineTiles : 0); }
inline TileShape tile_shape(int p, int t) { return t < kNumTiles ? kTiles[p][t] : kLineTiles[p][t - kNumTiles]; }

// Reference-element tables for one degree p, in the stage precision T.
template <typename T>
struct Tables {
  T w[kMaxN];             // Gauss-Lobatto weights on [0,1]
  T D[kMaxN * kMaxN];     // (D_1D)_{ij} = w_i phi_j'(xi_i), row-major
  T xi[kMaxN];            // Gauss-Lobatto points on [0,1] (node positions)
  T Vinv[kMaxN * kMaxN];  // nodal -> Legendre modal coefficients, row k = degree
  T nrm[kMaxN];           // squared L2 norm of L_k(2x-1) on [0,1]
};

// Smoothness indicator of Sec. 4.4 (off when on == 0): relaxed bounds of the limited field.
template <typename T>
struct SmoothnessT {
  int on;
  T s0, kappa, gmin, gmax;
};

// Per-stage statistics, reduced with atomics (non-negative floats stored as bit patterns).
struct StageStats {
  unsigned long long max_bound_violation;   // double bits
  unsigned long long max_entropy_violation; // double bits
  unsigned int rootfind_max_iters;
  unsigned int pad;
  unsigned long long rootfind_cap_hits;
  double field_scale;  // max |u| of the limited field at the last host set_state (violation floor)
  unsigned long long bound_nudges;  // float32 results set onto their bound by the post-round acceptance
};

// Moving two-state ghost of one side (the boundaries of the double Mach reflection, Sec. 5.7): the
// ghost state is a where the coordinate along the side (y on W/E, x on S/N) is below
// s0 + speed t (t the stage time), else b, or the mirrored trace (a slip wall) when wall_b.
template <typename T>
struct SplitBC {
  double s0, speed;
  T a[4], b[4];
  int wall_b;
  int set;  // 0 until sidp_set_split_boundary: the side then behaves as outflow
};

// One problem instance as seen by the kernels.
template <typename T>
struct Instance {
  const T* uin;      // stage input state, [nc][N]
  const T* u0;       // u^n (RK combination), [nc][N]
  T* uout;           // stage output, [nc][N]
  const T* ghost[4]; // exact-state ghost traces [nc][n_side*(p+1)] (or null)
  const double* dt;  // device scalar (float64 copy, for the clock and the host)
  const T* dtT;      // the same dt in the stage precision
  long long N;       // nodes per field
  int nx, ny;
  int bc[4];
  double h;
  T hT;              // h in the stage precision
  T x0, y0;          // lower-left corner of the domain (node positions)
  T c0, c1;          // RK combination uout = c0 u0 + c1 FE(uin)
  const SplitBC<T>* split;  // per side (split sides only), or null
  const T* geo;             // curved mesh: the per-node metric arrays [kGeoFields][N], or null (Cartesian)
  const double* tnow;       // time base of the launch (device scalar)
  double ck;                // stage time = *tnow + ck * dt
  // debug outputs (null = off), per node
  double* dbg_lo;
  double* dbg_hi;
  double* dbg_K;
  double* dbg_alpha;
  StageStats* stats; // null = off
};

// A launch over many instances: CTA i runs tasks[i] = (instance index, tile index); all tasks
// share degree, tile shape, law, precision and limiter.
template <typename T>
struct BatchLaunch {
  const Instance<T>* insts;  // device array, one per instance
  int stats;                 // the instances' statistics are on (launch the statistics kernels)
  const int2* tasks;         // device array of (instance, linear tile index)
  int ntasks;
  Tables<T> tab;
  LawParamsT<T> lp;
  int limiter;
  SmoothnessT<T> si;
  unsigned long long* bits;  // per-instance time-step accumulators (dt launches)
  int curved;                // the instances are on curved meshes: tasks are (instance, element block)
};

// A launch over every degree group at once (the single-launch batch mode): CTA i runs
// tasks[i] = (instance, linear tile index, degree p, 0) with the default tile shape of p; the
// reference tables of degree p are tabs[p] (device array, entries 1..kMaxP).  Subcell limiting
// without the smoothness indicator only.
template <typename T>
struct BatchAllLaunch {
  const Instance<T>* insts;
  const int4* tasks;
  int ntasks;
  const Tables<T>* tabs;
  LawParamsT<T> lp;
  SmoothnessT<T> si;         // off
  unsigned long long* bits;  // per-instance time-step accumulators (time-step launch)
};

template <typename T>
struct StageLaunch {
  Instance<T> inst;
  Tables<T> tab;
  LawParamsT<T> lp;
  int limiter;
  int dense;  // unsparsified graph viscosity (Sec. 3.4 comparison mode)
  SmoothnessT<T> si;
};

template <typename T>
inline SmoothnessT<T> make_smoothness(const sidp_config& c) {
  SmoothnessT<T> s{};
  s.on = c.smoothness ? 1 : 0;
  s.s0 = T(c.si_s0 != 0.0 ? c.si_s0 : -4.0 * std::log10((double)c.p));
  s.kappa = T(c.si_kappa > 0.0 ? c.si_kappa : 1.0);
  s.gmin = T(c.si_gmin);
  s.gmax = T(c.si_gmax);
  return s;
}

// Host-side helpers shared by the single-instance and batched entry points.
int tuned_tile(int law, int p, int mixed);  // autotuned tile index, or -1 when not tuned yet
sidp_status validate_config(const sidp_config* cfg, std::string& msg);
void set_last_error(const std::string& msg);  // the message sidp_last_error(NULL) returns

// Host tables (float64), computed once.
void gll_tables(int p, double* xi, double* w, double* D);
// Metric arrays of a curved mesh (sidp_geometry.cpp): kGeoFields x N values into out.
sidp_status curved_metrics(int p, int nx, int ny, const int* bc, const double* x, const double* y, double* out,
                           std::string& msg);
void modal_tables(int p, double* Vinv, double* nrm);

}  // namespace sidp

namespace sidp {
// Launcher of the stage kernel (dt_bits == nullptr) or the time-step kernel (dt_bits != nullptr)
// for one law, precision and degree with tile shape kTiles[P][tile]; explicitly specialised in
// the inst_<law>_<precision>*.cu translation units.
template <int LAW, typename T, int P>
cudaError_t launch_p(int tile, const StageLaunch<T>& a, unsigned long long* dt_bits, cudaStream_t s);
template <int LAW, typename T, int P>
cudaError_t launch_batch_p(int tile, const BatchLaunch<T>& b, bool dt, cudaStream_t s);
#define SIDP_DECLARE_P(LAWID, TT, P) \
  template <> cudaError_t launch_p<LAWID, TT, P>(int, const StageLaunch<TT>&, unsigned long long*, cudaStream_t); \
  template <> cudaError_t launch_batch_p<LAWID, TT, P>(int, const BatchLaunch<TT>&, bool, cudaStream_t);
#define SIDP_DECLARE(LAWID, TT) \
  SIDP_DECLARE_P(LAWID, TT, 1) SIDP_DECLARE_P(LAWID, TT, 2) SIDP_DECLARE_P(LAWID, TT, 3) SIDP_DECLARE_P(LAWID, TT, 4) \
  SIDP_DECLARE_P(LAWID, TT, 5) SIDP_DECLARE_P(LAWID, TT, 6) SIDP_DECLARE_P(LAWID, TT, 7)
SIDP_DECLARE(LAW_BURGERS, double)
SIDP_DECLARE(LAW_BURGERS, float)
SIDP_DECLARE(LAW_EULER, double)
SIDP_DECLARE(LAW_EULER, float)
SIDP_DECLARE(LAW_ADVECTION, double)
SIDP_DECLARE(LAW_ADVECTION, float)
SIDP_DECLARE(LAW_ADVECTION_VAR, double)
SIDP_DECLARE(LAW_ADVECTION_VAR, float)
#undef SIDP_DECLARE
#undef SIDP_DECLARE_P
// The single-launch batch kernels of one law and precision (inst_batch_all_*.cu) and their
// shared-memory size.
template <int LAW, typename T>
cudaError_t launch_batch_all(const BatchAllLaunch<T>& b, bool dt, cudaStream_t s);
#define SIDP_DECLARE_ALL(LAWID, TT) \
  template <> cudaError_t launch_batch_all<LAWID, TT>(const BatchAllLaunch<TT>&, bool, cudaStream_t);
SIDP_DECLARE_ALL(LAW_BURGERS, double)
SIDP_DECLARE_ALL(LAW_BURGERS, float)
SIDP_DECLARE_ALL(LAW_EULER, double)
SIDP_DECLARE_ALL(LAW_EULER, float)
SIDP_DECLARE_ALL(LAW_ADVECTION, double)
SIDP_DECLARE_ALL(LAW_ADVECTION, float)
SIDP_DECLARE_ALL(LAW_ADVECTION_VAR, double)
SIDP_DECLARE_ALL(LAW_ADVECTION_VAR, float)
#undef SIDP_DECLARE_ALL

// Instantiate launch_p for one law/precision/degree (used by the inst_*.cu files).
#define SIDP_INSTANTIATE_P(LAWID, LAWTPL, TT, P)                                                       \
  template <>                                                                                          \
  cudaError_t launch_p<LAWID, TT, P>(int tile, const StageLaunch<TT>& a, unsigned long long* bits,     \
                                     cudaStream_t s) {                                                 \
    if (a.inst.geo) { /* curved mesh: its own kernels (node layout; line layout for Euler) */           \
      if (tile >= kNumTiles && !bits && a.limiter == 2 && !a.si.on)                                    \
        return CurvedLines<P, LAWTPL<TT>, TT>::stage(a, a.inst.stats != nullptr, s);                   \
      return launch_curved<P, LAWTPL<TT>, TT>(a, bits, s);                                             \
    }                                                                                                  \
    if (a.dense) { /* unsparsified comparison mode: its own kernels, default tile shape */             \
      if (bits || a.limiter != 3)                                                                      \
        return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, false, true>(a, bits, s); \
      return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, true, true>(a, bits, s);  \
    }                                                                                                  \
    if (a.limiter == 3 && !bits) /* elementwise limiting: its own kernel, default tile shape */       \
      return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, true>(a, bits, s);       \
    if (tile >= kNumTiles && !bits && a.limiter == 2 && !a.si.on) /* the line kernel (and its statistics variant) */ \
      return LineDispatch<LAWID, P, LAWTPL<TT>, TT>::stage(tile - kNumTiles, a, a.inst.stats != nullptr, s); \
    if (tile >= kNumTiles && bits) /* the time step on the line kernel's tiles */                     \
      return LineDispatch<LAWID, P, LAWTPL<TT>, TT>::dt(tile - kNumTiles, a, bits, s);                  \
    if (a.inst.stats && !bits) /* statistics on: the statistics kernel, default tile shape */         \
      return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, false, false, true>(a, bits, s); \
    if (!bits && (a.limiter != 2 || a.si.on)) /* other modes: the general kernel, default tile shape */ \
      return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT>(a, bits, s);             \
    switch (tile < kNumTiles ? tile : 0) { /* subcell limiting without the indicator (and the time step): every tile shape */ \
      case 0: return launch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, false, false, false, true>(a, bits, s); \
      case 1: return launch_tile<P, kTiles[P][1].tx, kTiles[P][1].ty, LAWTPL<TT>, TT, false, false, false, true>(a, bits, s); \
      case 2: return launch_tile<P, kTiles[P][2].tx, kTiles[P][2].ty, LAWTPL<TT>, TT, false, false, false, true>(a, bits, s); \
      case 3: return launch_tile<P, kTiles[P][3].tx, kTiles[P][3].ty, LAWTPL<TT>, TT, false, false, false, true>(a, bits, s); \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t launch_batch_p<LAWID, TT, P>(int tile, const BatchLaunch<TT>& b, bool dt, cudaStream_t s) { \
    if (b.curved) /* curved meshes: their own kernels */                                              \
      return launch_curved_batch<P, LAWTPL<TT>, TT>(b, dt, s);                                         \
    if (tile >= kNumTiles && !dt && b.limiter == 2 && !b.si.on) /* the line kernel */                 \
      return LineDispatch<LAWID, P, LAWTPL<TT>, TT>::batch(tile - kNumTiles, b, b.stats != 0, s);      \
    if (b.limiter == 3 && !dt)                                                                         \
      return launch_batch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, true>(b, dt, s);  \
    if (b.stats && !dt)                                                                                \
      return launch_batch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, false, true>(b, dt, s); \
    if (!dt && (b.limiter != 2 || b.si.on))                                                            \
      return launch_batch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT>(b, dt, s);         \
    switch (tile < kNumTiles ? tile : 0) {                                                             \
      case 0: return launch_batch_tile<P, kTiles[P][0].tx, kTiles[P][0].ty, LAWTPL<TT>, TT, false, false, true>(b, dt, s); \
      case 1: return launch_batch_tile<P, kTiles[P][1].tx, kTiles[P][1].ty, LAWTPL<TT>, TT, false, false, true>(b, dt, s); \
      case 2: return launch_batch_tile<P, kTiles[P][2].tx, kTiles[P][2].ty, LAWTPL<TT>, TT, false, false, true>(b, dt, s); \
      case 3: return launch_batch_tile<P, kTiles[P][3].tx, kTiles[P][3].ty, LAWTPL<TT>, TT, false, false, true>(b, dt, s); \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
  }
}  // namespace sidp
