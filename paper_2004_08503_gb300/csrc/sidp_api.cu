// C-ABI of libsidp: contexts, state transfer, stages, steps (CUDA graph), diagnostics.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sidp.h"
#include "sidp_internal.h"

using namespace sidp;

namespace {

// ---------------------------------------------------------------- small kernels
// dt of an explicit stage call; stage 1 also takes the clock as the time base of the step.
__global__ void k_set_scalar(double* dst, double v, int step_start) {
  dst[0] = v;
  *reinterpret_cast<float*>(dst + 2) = (float)v;
  if (step_start) dst[3] = dst[1];
}

__global__ void k_set_time(double* dst, double t) {
  dst[1] = t;
  dst[3] = t;
}

// dt = cfl * min (Eq. cfl-low with the CFL constant); 0 when no wave moves; advances the clock
// and re-arms the min accumulator for the next step.
__global__ void k_dt_finalize(unsigned long long* bits, double cfl, double* dt, double* clock) {
  const double mn = __longlong_as_double((long long)*bits);
  const double v = (mn < DBL_MAX) ? cfl * mn : 0.0;
  dt[0] = v;
  *reinterpret_cast<float*>(dt + 2) = (float)v;
  if (clock) {
    dt[3] = *clock;  // t^n: the time base of the step's stages
    *clock += v;
  }
  *bits = (unsigned long long)__double_as_longlong(DBL_MAX);
}

constexpr int kDiagK = 15;  // mass[4], min[4], max[4], rho_min, p_min, nonfinite

template <typename T>
__global__ void k_diag_partial(const T* u, long long N, int nc, int n, double h, const double* wtab, double gamma,
                               int euler, const double* mnode, double* part) {
  double acc[kDiagK];
  for (int f = 0; f < 4; ++f) { acc[f] = 0.0; acc[4 + f] = DBL_MAX; acc[8 + f] = -DBL_MAX; }
  acc[12] = DBL_MAX; acc[13] = DBL_MAX; acc[14] = 0.0;
  const int NN = n * n;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(g % NN), a = node / n, b = node % n;
    const double m = mnode ? mnode[g] : h * h * wtab[a] * wtab[b];
    double v[4] = {0, 0, 0, 0};
    for (int f = 0; f < nc; ++f) {
      v[f] = (double)u[f * N + g];
      if (!isfinite(v[f])) { acc[14] += 1.0; continue; }
      acc[f] += m * v[f];
      acc[4 + f] = fmin(acc[4 + f], v[f]);
      acc[8 + f] = fmax(acc[8 + f], v[f]);
    }
    if (euler) {
      const double p = (gamma - 1.0) * (v[3] - 0.5 * (v[1] * v[1] + v[2] * v[2]) / v[0]);
      acc[12] = fmin(acc[12], v[0]);
      acc[13] = fmin(acc[13], p);
    }
  }
  __shared__ double red[kDiagK][256];
  for (int k = 0; k < kDiagK; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      for (int k = 0; k < kDiagK; ++k) {
        const double x = red[k][threadIdx.x], y = red[k][threadIdx.x + s];
        red[k][threadIdx.x] = (k < 4 || k == 14) ? x + y : ((k >= 8 && k < 12) ? fmax(x, y) : fmin(x, y));
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < kDiagK; ++k) part[blockIdx.x * kDiagK + k] = red[k][0];
}

__global__ void k_diag_final(const double* part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double acc[kDiagK];
  for (int k = 0; k < kDiagK; ++k) acc[k] = part[k];
  for (int bi = 1; bi < nb; ++bi)
    for (int k = 0; k < kDiagK; ++k) {
      const double y = part[bi * kDiagK + k];
      acc[k] = (k < 4 || k == 14) ? acc[k] + y : ((k >= 8 && k < 12) ? fmax(acc[k], y) : fmin(acc[k], y));
    }
  for (int k = 0; k < kDiagK; ++k) out[k] = acc[k];
}

constexpr int kDiagBlocks = 256;

const char* kStatusStr[] = {"ok", "invalid argument", "CUDA error", "non-finite state", "inadmissible state",
                            "entropy line search iteration cap", "call out of order", "device allocation failed"};

thread_local std::string g_last_error;

}  // namespace

namespace sidp {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace sidp

struct sidp_ctx {
  sidp_config cfg{};
  int n = 0, NN = 0, nc = 0;
  long long Ne = 0, N = 0;
  double h = 0;
  bool mixed = false;
  size_t esize = 8;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* d_u[3] = {nullptr, nullptr, nullptr};  // u^n, u^(1), u^(2)
  void* d_ghost[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d_scal = nullptr;  // [0] dt, [1] clock, [2] dt as float32, [3] time at the step's start
  void* d_split = nullptr;   // SplitBC<T>[4]
  unsigned long long* d_bits = nullptr;
  StageStats* d_stats = nullptr;
  double* d_dbg = nullptr;  // 4 * N
  double* d_wtab = nullptr;
  double* d_part = nullptr;
  double* d_diag = nullptr;
  void* d_geo = nullptr;     // curved mesh: [kGeoFields][N] in the stage precision
  double* d_mass = nullptr;  // curved mesh: m_i in float64 (diagnostics)
  bool curved = false;
  std::vector<double> hx, hy;  // curved mesh: node coordinates
  bool debug = false, stats_on = true, use_graph = true;
  int stage_done = 0;
  long long steps = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_warm = false;
  int tile = 0;          // tile candidate: kTiles[p][tile] (< kNumTiles), else a line-kernel tile
  bool tuned = false;
  bool settle = false;      // a second autotuner pass is due at settle_at steps
  long long settle_at = 0;
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  std::string err;
};

namespace {

sidp_status fail(sidp_ctx* c, sidp_status s, const std::string& msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return s;
}

#define CUDA_TRY(ctx, expr)                                                                          \
  do {                                                                                               \
    cudaError_t _e = (expr);                                                                         \
    if (_e != cudaSuccess)                                                                           \
      return fail(ctx, SIDP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));         \
  } while (0)

// d_scal layout: [0] dt (float64), [1] simulated time, [2] dt as float32 (low 4 bytes), [3] t^n
template <typename T> const T* dt_ptr(const sidp_ctx* c);
template <> const double* dt_ptr<double>(const sidp_ctx* c) { return c->d_scal; }
template <> const float* dt_ptr<float>(const sidp_ctx* c) { return reinterpret_cast<const float*>(c->d_scal + 2); }

template <typename T>
void fill_launch(const sidp_ctx* c, StageLaunch<T>& L) {
  std::memset(&L, 0, sizeof(L));
  L.inst.N = c->N;
  L.inst.nx = c->cfg.nx;
  L.inst.ny = c->cfg.ny;
  for (int s = 0; s < 4; ++s) {
    L.inst.bc[s] = c->cfg.bc[s];
    L.inst.ghost[s] = static_cast<const T*>(c->d_ghost[s]);
  }
  L.inst.h = c->h;
  L.inst.hT = T(c->h);
  L.inst.x0 = T(c->cfg.x0);
  L.inst.y0 = T(c->cfg.y0);
  L.inst.dt = c->d_scal;
  L.inst.split = static_cast<const SplitBC<T>*>(c->d_split);
  L.inst.tnow = c->d_scal + 3;
  L.inst.ck = 0.0;
  L.inst.dtT = dt_ptr<T>(c);
  L.inst.geo = static_cast<const T*>(c->d_geo);
  for (int i = 0; i < c->n; ++i) { L.tab.w[i] = T(c->w[i]); L.tab.xi[i] = T(c->xi[i]); }
  for (int i = 0; i < c->n * c->n; ++i) L.tab.D[i] = T(c->D[i]);
  L.lp = make_law_params<T>(c->cfg.gamma, c->cfg.adv_beta, c->cfg.adv_grad);
  {
    double Vinv[kMaxN * kMaxN], nrm[kMaxN];
    modal_tables(c->cfg.p, Vinv, nrm);
    for (int i = 0; i < c->n * c->n; ++i) L.tab.Vinv[i] = T(Vinv[i]);
    for (int i = 0; i < c->n; ++i) L.tab.nrm[i] = T(nrm[i]);
    L.si = make_smoothness<T>(c->cfg);
  }
  L.limiter = c->cfg.limiter;
  L.dense = c->cfg.unsparsified;
  if (c->debug) {
    L.inst.dbg_lo = c->d_dbg;
    L.inst.dbg_hi = c->d_dbg + c->N;
    L.inst.dbg_K = c->d_dbg + 2 * c->N;
    L.inst.dbg_alpha = c->d_dbg + 3 * c->N;
  }
  L.inst.stats = c->stats_on ? c->d_stats : nullptr;
}

template <int LAW, typename T>
cudaError_t launch_law(int p, int tile, const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s) {
  switch (p) {
    case 1: return launch_p<LAW, T, 1>(tile, a, bits, s);
    case 2: return launch_p<LAW, T, 2>(tile, a, bits, s);
    case 3: return launch_p<LAW, T, 3>(tile, a, bits, s);
    case 4: return launch_p<LAW, T, 4>(tile, a, bits, s);
    case 5: return launch_p<LAW, T, 5>(tile, a, bits, s);
    case 6: return launch_p<LAW, T, 6>(tile, a, bits, s);
    case 7: return launch_p<LAW, T, 7>(tile, a, bits, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t dispatch(int law, int p, int tile, const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s) {
  switch (law) {
    case LAW_BURGERS: return launch_law<LAW_BURGERS, T>(p, tile, a, bits, s);
    case LAW_EULER: return launch_law<LAW_EULER, T>(p, tile, a, bits, s);
    case LAW_ADVECTION: return launch_law<LAW_ADVECTION, T>(p, tile, a, bits, s);
    case LAW_ADVECTION_VAR: return launch_law<LAW_ADVECTION_VAR, T>(p, tile, a, bits, s);
    default: return cudaErrorInvalidValue;
  }
}

// Stage k of SSP-RK3 (Sec. 5) on the device buffers of the context.
template <typename T>
cudaError_t run_stage_t(sidp_ctx* c, int k) {
  StageLaunch<T> L;
  fill_launch(c, L);
  T* un = static_cast<T*>(c->d_u[0]);
  T* u1 = static_cast<T*>(c->d_u[1]);
  T* u2 = static_cast<T*>(c->d_u[2]);
  if (k == 1) { L.inst.uin = un; L.inst.u0 = un; L.inst.uout = u1; L.inst.c0 = T(0); L.inst.c1 = T(1); }
  else if (k == 2) { L.inst.uin = u1; L.inst.u0 = un; L.inst.uout = u2; L.inst.c0 = T(0.75); L.inst.c1 = T(0.25); }
  else { L.inst.uin = u2; L.inst.u0 = un; L.inst.uout = un; L.inst.c0 = T(1.0 / 3.0); L.inst.c1 = T(2.0 / 3.0); }
  L.inst.ck = (k == 1) ? 0.0 : (k == 2) ? 1.0 : 0.5;  // SSP-RK3 stage times t^n + ck dt
  return dispatch<T>(c->cfg.law, c->cfg.p, c->tile, L, nullptr, c->stream);
}

cudaError_t run_stage(sidp_ctx* c, int k) { return c->mixed ? run_stage_t<float>(c, k) : run_stage_t<double>(c, k); }

template <typename T>
cudaError_t run_dt_t(sidp_ctx* c, bool advance_clock) {
  StageLaunch<T> L;
  fill_launch(c, L);
  L.inst.uin = static_cast<const T*>(c->d_u[0]);
  L.inst.tnow = c->d_scal + 1;  // the time step is taken at t^n (the clock before it advances)
  cudaError_t e = dispatch<T>(c->cfg.law, c->cfg.p, c->tile, L, c->d_bits, c->stream);
  if (e != cudaSuccess) return e;
  k_dt_finalize<<<1, 1, 0, c->stream>>>(c->d_bits, c->cfg.cfl, c->d_scal, advance_clock ? c->d_scal + 1 : nullptr);
  return cudaGetLastError();
}

cudaError_t run_dt(sidp_ctx* c, bool adv) { return c->mixed ? run_dt_t<float>(c, adv) : run_dt_t<double>(c, adv); }

cudaError_t run_step(sidp_ctx* c) {
  cudaError_t e = run_dt(c, true);
  for (int k = 1; k <= 3 && e == cudaSuccess; ++k) e = run_stage(c, k);
  return e;
}

// ---------------------------------------------------------------- tile autotuner
// Picks the stage kernel's tile candidate per (law, p, precision, curved or not) by timing stage 1
// of every candidate on the context's current state: node-layout tiles kTiles[p] and, for Euler,
// line-layout tiles kLineTiles[p] (on a curved mesh: the node layout and the line layout).  Two
// passes: at the first step, and once more at kSettleSteps steps, whose choice is kept for the
// process.  Results differ between the layouts only in the rounding of sums.  SIDP_TILE=<i>
// forces a candidate, SIDP_AUTOTUNE=0 keeps the default; SIDP_TUNE_FILE=<path> loads and stores
// the settled table ("law p slot tile" lines, slot = precision (0 float64, 1 mixed) + 2 on a
// curved mesh).
std::mutex g_tune_mu;
// last index: precision (0 float64, 1 mixed) + 2 on curved meshes
int g_tune[LAW_ADVECTION_VAR + 1][kMaxP + 1][4];
bool g_settled[LAW_ADVECTION_VAR + 1][kMaxP + 1][4];  // chosen by the second pass (or loaded from a file)
bool g_tune_init = false;
// The first steps of a flow (a blast's initial transient, say) can favour another tile than the
// rest of the run: the autotuner times the candidates at the first step and once more at this step.
constexpr long long kSettleSteps = 10;

void tune_table_init() {
  if (g_tune_init) return;
  for (auto& a : g_tune)
    for (auto& b : a) b[0] = b[1] = b[2] = b[3] = -1;
  for (auto& a : g_settled)
    for (auto& b : a) b[0] = b[1] = b[2] = b[3] = false;
  if (const char* f = std::getenv("SIDP_TUNE_FILE")) {
    if (FILE* fp = std::fopen(f, "r")) {
      int law, p, mixed, tile;
      while (std::fscanf(fp, "%d %d %d %d", &law, &p, &mixed, &tile) == 4)
        if (law >= 1 && law <= 3 && p >= 1 && p <= kMaxP && mixed >= 0 && mixed <= 3 && tile >= 0 &&
            tile < num_tile_candidates(law)) {
          g_tune[law][p][mixed] = tile;
          g_settled[law][p][mixed] = true;
        }
      std::fclose(fp);
    }
  }
  g_tune_init = true;
}

void tune_table_store() {
  const char* f = std::getenv("SIDP_TUNE_FILE");
  if (!f) return;
  if (FILE* fp = std::fopen(f, "w")) {
    for (int law = 1; law <= 3; ++law)
      for (int p = 1; p <= kMaxP; ++p)
        for (int m = 0; m < 4; ++m)
          if (g_tune[law][p][m] >= 0) std::fprintf(fp, "%d %d %d %d\n", law, p, m, g_tune[law][p][m]);
    std::fclose(fp);
  }
}

cudaError_t run_stage(sidp_ctx* c, int k);
cudaError_t run_dt(sidp_ctx* c, bool adv);
}  // namespace

namespace sidp {
int tuned_tile(int law, int p, int mixed) {
  if (const char* f = std::getenv("SIDP_TILE")) {
    const int t = std::atoi(f);
    if (t >= 0 && t < num_tile_candidates(law)) return t;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_table_init();
  if (law < 1 || law > LAW_ADVECTION_VAR || p < 1 || p > kMaxP || mixed < 0 || mixed > 1) return -1;
  return g_tune[law][p][mixed];
}
}  // namespace sidp

namespace {

// second: the second pass (at kSettleSteps steps), which times the candidates again whatever the
// table holds and marks the choice settled.
cudaError_t autotune(sidp_ctx* c, bool second = false) {
  if (c->tuned && !second) return cudaSuccess;
  c->tuned = true;
  c->settle = false;
  // only subcell limiting without the smoothness indicator has a stage kernel for every shape;
  // the other modes run the default one
  if (c->cfg.limiter != 2 || c->cfg.smoothness) { c->tile = 0; return cudaSuccess; }
  if (const char* f = std::getenv("SIDP_TILE")) {
    const int t = std::atoi(f);
    if (t >= 0 && t < num_tile_candidates(c->cfg.law)) c->tile = t;
    return cudaSuccess;
  }
  const char* off = std::getenv("SIDP_AUTOTUNE");
  if (off && off[0] == '0') return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_table_init();
  const int ti = (c->mixed ? 1 : 0) + (c->curved ? 2 : 0);
  int& slot = g_tune[c->cfg.law][c->cfg.p][ti];
  bool& settled = g_settled[c->cfg.law][c->cfg.p][ti];
  if (slot >= 0 && (settled || !second)) {
    c->tile = slot;
    if (!settled) { c->settle = true; c->settle_at = c->steps + kSettleSteps; }
    return cudaSuccess;
  }
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  if ((err = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return err; }
  float best = 1e30f;
  int best_t = 0;
  const int saved = c->tile;
  // candidates: every tile of both layouts on a Cartesian mesh; on a curved mesh the node layout
  // (0) and, for Euler, the line layout (kNumTiles)
  int cand[kMaxCand], ncand = 0;
  if (c->curved) {
    cand[ncand++] = 0;
    if (c->cfg.law == LAW_EULER) cand[ncand++] = kNumTiles;
  } else {
    for (int t = 0; t < num_tile_candidates(c->cfg.law); ++t) cand[ncand++] = t;
  }
  for (int ci = 0; ci < ncand && err == cudaSuccess; ++ci) {
    const int t = cand[ci];
    c->tile = t;
    if ((err = run_dt(c, false)) != cudaSuccess) break;
    if ((err = run_stage(c, 1)) != cudaSuccess) break;  // warm-up (and kernel attributes)
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run_stage(c, 1);
    cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best) { best = ms; best_t = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) { c->tile = saved; return err; }
  c->tile = best_t;
  slot = best_t;
  settled = second;
  if (!second) { c->settle = true; c->settle_at = c->steps + kSettleSteps; }
  if (second) tune_table_store();
  return cudaSuccess;
}

void drop_graph(sidp_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

}  // namespace

namespace sidp {
sidp_status validate_config(const sidp_config* cfg, std::string& msg) {
  if (!cfg) { msg = "null config"; return SIDP_ERR_ARG; }
  if (cfg->law != SIDP_LAW_BURGERS2D && cfg->law != SIDP_LAW_EULER2D && cfg->law != SIDP_LAW_ADVECTION2D &&
      cfg->law != SIDP_LAW_ADVECTION_VAR2D) { msg = "unknown law"; return SIDP_ERR_ARG; }
  if (cfg->p < 1 || cfg->p > kMaxP) { msg = "p must be in 1..7"; return SIDP_ERR_ARG; }
  if (cfg->nx < 1 || cfg->ny < 1) { msg = "nx, ny must be >= 1"; return SIDP_ERR_ARG; }
  if ((long long)cfg->nx * cfg->ny > 2147483647LL) { msg = "a mesh has fewer than 2^31 elements"; return SIDP_ERR_ARG; }
  if (cfg->precision != SIDP_FP64 && cfg->precision != SIDP_MIXED) { msg = "unknown precision"; return SIDP_ERR_ARG; }
  const double hx = (cfg->x1 - cfg->x0) / cfg->nx, hy = (cfg->y1 - cfg->y0) / cfg->ny;
  if (!(hx > 0) || !(hy > 0) || std::fabs(hx - hy) > 1e-12 * hx) { msg = "elements must be square with positive size"; return SIDP_ERR_ARG; }
  for (int s = 0; s < 4; ++s) {
    if (cfg->bc[s] < 0 || cfg->bc[s] > 4) { msg = "unknown boundary condition"; return SIDP_ERR_ARG; }
    if (cfg->bc[s] == SIDP_BC_SLIP_WALL && cfg->law != SIDP_LAW_EULER2D) { msg = "slip walls need the Euler law"; return SIDP_ERR_ARG; }
  }
  if ((cfg->bc[0] == SIDP_BC_PERIODIC) != (cfg->bc[1] == SIDP_BC_PERIODIC) ||
      (cfg->bc[2] == SIDP_BC_PERIODIC) != (cfg->bc[3] == SIDP_BC_PERIODIC)) { msg = "periodic sides must be paired"; return SIDP_ERR_ARG; }
  if (!(cfg->cfl > 0.0) || cfg->cfl > 1.0) { msg = "cfl must be in (0,1]"; return SIDP_ERR_ARG; }
  if (cfg->law == SIDP_LAW_EULER2D && !(cfg->gamma > 1.0 && cfg->gamma <= 5.0 / 3.0)) { msg = "gamma must be in (1, 5/3]"; return SIDP_ERR_ARG; }
  if (cfg->limiter < 0 || cfg->limiter > 3) { msg = "unknown limiter"; return SIDP_ERR_ARG; }
  if (!std::isfinite(cfg->adv_beta[0]) || !std::isfinite(cfg->adv_beta[1])) { msg = "non-finite advection velocity"; return SIDP_ERR_ARG; }
  if (cfg->law == SIDP_LAW_ADVECTION_VAR2D && (!std::isfinite(cfg->adv_grad[0]) || !std::isfinite(cfg->adv_grad[1]))) {
    msg = "non-finite advection velocity gradient"; return SIDP_ERR_ARG;
  }
  if (cfg->smoothness != 0 && cfg->smoothness != 1) { msg = "smoothness must be 0 or 1"; return SIDP_ERR_ARG; }
  if (cfg->unsparsified != 0 && cfg->unsparsified != 1) { msg = "unsparsified must be 0 or 1"; return SIDP_ERR_ARG; }
  if (cfg->smoothness && (!std::isfinite(cfg->si_gmin) || !std::isfinite(cfg->si_gmax) || cfg->si_gmin > cfg->si_gmax ||
                          !std::isfinite(cfg->si_s0) || !std::isfinite(cfg->si_kappa))) {
    msg = "smoothness indicator needs finite s0, kappa and g_min <= g_max"; return SIDP_ERR_ARG;
  }
  return SIDP_OK;
}
}  // namespace sidp

namespace {

template <typename T>
sidp_status upload(sidp_ctx* c, void* dst, const double* src, long long count) {
  std::vector<T> tmp(count);
  for (long long i = 0; i < count; ++i) tmp[i] = T(src[i]);
  CUDA_TRY(c, cudaMemcpyAsync(dst, tmp.data(), count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return SIDP_OK;
}

template <typename T>
sidp_status download(sidp_ctx* c, const void* src, double* dst, long long count) {
  std::vector<T> tmp(count);
  CUDA_TRY(c, cudaMemcpyAsync(tmp.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (long long i = 0; i < count; ++i) dst[i] = double(tmp[i]);
  return SIDP_OK;
}

}  // namespace

namespace {
template <typename T>
SplitBC<T> make_split(double s0, double speed, const double* a, const double* b, int nc) {
  SplitBC<T> sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.s0 = s0;
  sp.speed = speed;
  for (int f = 0; f < nc; ++f) {
    sp.a[f] = T(a[f]);
    sp.b[f] = b ? T(b[f]) : T(0);
  }
  sp.wall_b = b ? 0 : 1;
  sp.set = 1;
  return sp;
}
}  // namespace

extern "C" {

const char* sidp_status_str(sidp_status s) {
  const int i = (int)s;
  return (i >= 0 && i < (int)(sizeof(kStatusStr) / sizeof(kStatusStr[0]))) ? kStatusStr[i] : "unknown status";
}

const char* sidp_last_error(const sidp_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

sidp_status sidp_create(sidp_ctx** out, const sidp_config* cfg, void* cuda_stream) try {
  if (!out) return fail(nullptr, SIDP_ERR_ARG, "null output pointer");
  *out = nullptr;
  std::string msg;
  sidp_status st = validate_config(cfg, msg);
  if (st != SIDP_OK) return fail(nullptr, st, msg);
  sidp_ctx* c = new sidp_ctx();
  c->cfg = *cfg;
  c->n = cfg->p + 1;
  c->NN = c->n * c->n;
  c->nc = (cfg->law == SIDP_LAW_EULER2D) ? 4 : 1;
  c->Ne = (long long)cfg->nx * cfg->ny;
  c->N = c->Ne * c->NN;
  c->h = (cfg->x1 - cfg->x0) / cfg->nx;
  c->mixed = cfg->precision == SIDP_MIXED;
  c->esize = c->mixed ? 4 : 8;
  gll_tables(cfg->p, c->xi, c->w, c->D);
  auto bail = [&](sidp_status s, const std::string& m) {
    g_last_error = m;
    sidp_destroy(c);
    return s;
  };
  cudaError_t e;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
    c->own_stream = true;
  }
  const size_t bytes = (size_t)c->nc * c->N * c->esize;
  for (int i = 0; i < 3; ++i)
    if (cudaMalloc(&c->d_u[i], bytes) != cudaSuccess) return bail(SIDP_ERR_OOM, "state allocation failed");
  if (cudaMalloc(&c->d_scal, 4 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_bits, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->d_stats, sizeof(StageStats)) != cudaSuccess ||
      cudaMalloc(&c->d_wtab, kMaxN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_part, kDiagBlocks * kDiagK * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_diag, kDiagK * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_split, 4 * (c->mixed ? sizeof(SplitBC<float>) : sizeof(SplitBC<double>))) != cudaSuccess)
    return bail(SIDP_ERR_OOM, "scratch allocation failed");
  double zero2[4] = {0.0, 0.0, 0.0, 0.0};
  const unsigned long long big = (unsigned long long)0x7fefffffffffffffULL;  // DBL_MAX bits
  StageStats zs{};
  if ((e = cudaMemcpy(c->d_scal, zero2, sizeof(zero2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_bits, &big, sizeof(big), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_stats, &zs, sizeof(zs), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_wtab, c->w, kMaxN * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(c->d_u[0], 0, bytes)) != cudaSuccess ||
      (e = cudaMemset(c->d_split, 0, 4 * (c->mixed ? sizeof(SplitBC<float>) : sizeof(SplitBC<double>)))) != cudaSuccess)
    return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  *out = c;
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(nullptr, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(nullptr, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_destroy(sidp_ctx* c) {
  if (!c) return SIDP_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  for (int i = 0; i < 3; ++i) cudaFree(c->d_u[i]);
  for (int s = 0; s < 4; ++s) cudaFree(c->d_ghost[s]);
  cudaFree(c->d_scal);
  cudaFree(c->d_split);
  cudaFree(c->d_bits);
  cudaFree(c->d_stats);
  cudaFree(c->d_dbg);
  cudaFree(c->d_wtab);
  cudaFree(c->d_part);
  cudaFree(c->d_diag);
  cudaFree(c->d_geo);
  cudaFree(c->d_mass);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return SIDP_OK;
}

sidp_status sidp_sizes(const sidp_ctx* c, long long* n_nodes, int* nc) {
  if (!c) return fail(nullptr, SIDP_ERR_ARG, "null context");
  if (n_nodes) *n_nodes = c->N;
  if (nc) *nc = c->nc;
  return SIDP_OK;
}

sidp_status sidp_node_coords(const sidp_ctx* c, double* x, double* y) {
  if (!c || !x || !y) return fail(nullptr, SIDP_ERR_ARG, "null argument");
  if (c->curved) {
    std::memcpy(x, c->hx.data(), c->N * sizeof(double));
    std::memcpy(y, c->hy.data(), c->N * sizeof(double));
    return SIDP_OK;
  }
  const int n = c->n;
  for (long long e = 0; e < c->Ne; ++e) {
    const long long ex = e % c->cfg.nx, ey = e / c->cfg.nx;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        const long long g = e * c->NN + a * n + b;
        x[g] = c->cfg.x0 + ((double)ex + c->xi[b]) * c->h;
        y[g] = c->cfg.y0 + ((double)ey + c->xi[a]) * c->h;
      }
  }
  return SIDP_OK;
}

sidp_status sidp_set_state(sidp_ctx* c, const double* u) try {
  if (!c || !u) return fail(c, SIDP_ERR_ARG, "null argument");
  const long long N = c->N;
  for (long long i = 0; i < c->nc * N; ++i)
    if (!std::isfinite(u[i])) return fail(c, SIDP_ERR_NONFINITE, "state holds a non-finite value");
  if (c->cfg.law == SIDP_LAW_EULER2D) {
    const double g = c->cfg.gamma;
    for (long long i = 0; i < N; ++i) {
      const double r = u[i], mx = u[N + i], my = u[2 * N + i], E = u[3 * N + i];
      const double p = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / r);
      if (!(r > 0) || !(p > 0)) return fail(c, SIDP_ERR_BOUNDS, "Euler state with rho <= 0 or p <= 0");
    }
  }
  sidp_status st = c->mixed ? upload<float>(c, c->d_u[0], u, c->nc * N) : upload<double>(c, c->d_u[0], u, c->nc * N);
  if (st != SIDP_OK) return st;
  StageStats zs{};
  for (long long i = 0; i < N; ++i) zs.field_scale = std::fmax(zs.field_scale, std::fabs(u[i]));
  CUDA_TRY(c, cudaMemcpy(c->d_stats, &zs, sizeof(zs), cudaMemcpyHostToDevice));
  c->stage_done = 0;
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_get_state(sidp_ctx* c, int which, double* u) try {
  if (!c || !u) return fail(c, SIDP_ERR_ARG, "null argument");
  if (which < 0 || which > 2) return fail(c, SIDP_ERR_ARG, "which must be 0, 1 or 2");
  return c->mixed ? download<float>(c, c->d_u[which], u, c->nc * c->N) : download<double>(c, c->d_u[which], u, c->nc * c->N);
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_upload_state(sidp_ctx* c, const void* host) {
  if (!c || !host) return fail(c, SIDP_ERR_ARG, "null argument");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_u[0], host, (size_t)c->nc * c->N * c->esize, cudaMemcpyHostToDevice, c->stream));
  c->stage_done = 0;
  return SIDP_OK;
}

sidp_status sidp_download_state(sidp_ctx* c, int which, void* host) {
  if (!c || !host) return fail(c, SIDP_ERR_ARG, "null argument");
  if (which < 0 || which > 2) return fail(c, SIDP_ERR_ARG, "which must be 0, 1 or 2");
  CUDA_TRY(c, cudaMemcpyAsync(host, c->d_u[which], (size_t)c->nc * c->N * c->esize, cudaMemcpyDeviceToHost, c->stream));
  return SIDP_OK;
}

sidp_status sidp_set_ghost_state(sidp_ctx* c, int side, const double* u) try {
  if (!c || !u || side < 0 || side > 3) return fail(c, SIDP_ERR_ARG, "bad argument");
  const long long nside = (side < 2) ? c->cfg.ny : c->cfg.nx;
  const long long count = c->nc * nside * c->n;
  if (!c->d_ghost[side]) {
    if (cudaMalloc(&c->d_ghost[side], count * c->esize) != cudaSuccess) return fail(c, SIDP_ERR_OOM, "ghost allocation failed");
    drop_graph(c);
  }
  return c->mixed ? upload<float>(c, c->d_ghost[side], u, count) : upload<double>(c, c->d_ghost[side], u, count);
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}


sidp_status sidp_set_split_boundary(sidp_ctx* c, int side, double s0, double speed, const double* state_a,
                                    const double* state_b) {
  if (!c || side < 0 || side > 3 || !state_a) return fail(c, SIDP_ERR_ARG, "bad argument");
  if (c->cfg.bc[side] != SIDP_BC_SPLIT) return fail(c, SIDP_ERR_STATE, "the side is not a split side");
  if (!state_b && c->cfg.law != SIDP_LAW_EULER2D) return fail(c, SIDP_ERR_ARG, "a slip-wall part needs the Euler law");
  if (std::isnan(s0) || !std::isfinite(speed)) return fail(c, SIDP_ERR_ARG, "split point must be a number, speed finite");
  for (int f = 0; f < c->nc; ++f)
    if (!std::isfinite(state_a[f]) || (state_b && !std::isfinite(state_b[f]))) return fail(c, SIDP_ERR_NONFINITE, "non-finite state");
  if (c->mixed) {
    const SplitBC<float> sp = make_split<float>(s0, speed, state_a, state_b, c->nc);
    CUDA_TRY(c, cudaMemcpy(static_cast<SplitBC<float>*>(c->d_split) + side, &sp, sizeof(sp), cudaMemcpyHostToDevice));
  } else {
    const SplitBC<double> sp = make_split<double>(s0, speed, state_a, state_b, c->nc);
    CUDA_TRY(c, cudaMemcpy(static_cast<SplitBC<double>*>(c->d_split) + side, &sp, sizeof(sp), cudaMemcpyHostToDevice));
  }
  return SIDP_OK;
}

sidp_status sidp_curved_metrics(int p, int nx, int ny, const int* bc, const double* x, const double* y,
                                double* out) try {
  std::string msg;
  const sidp_status st = curved_metrics(p, nx, ny, bc, x, y, out, msg);
  if (st != SIDP_OK) return fail(nullptr, st, msg);
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(nullptr, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(nullptr, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_set_geometry(sidp_ctx* c, const double* x, const double* y) try {
  if (!c || !x || !y) return fail(c, SIDP_ERR_ARG, "null argument");
  const sidp_config& f = c->cfg;
  if (f.law == SIDP_LAW_ADVECTION_VAR2D)
    return fail(c, SIDP_ERR_ARG, "variable-velocity advection is defined on Cartesian meshes only");
  if (f.unsparsified)
    return fail(c, SIDP_ERR_ARG, "curved meshes take no unsparsified mode");
  for (int k = 0; k < 4; ++k)
    if (f.bc[k] != SIDP_BC_PERIODIC && f.bc[k] != SIDP_BC_OUTFLOW && f.bc[k] != SIDP_BC_SLIP_WALL)
      return fail(c, SIDP_ERR_ARG, "curved meshes take periodic, outflow or slip-wall sides");
  std::vector<double> geo((size_t)kGeoFields * c->N);
  std::string msg;
  const sidp_status st = curved_metrics(f.p, f.nx, f.ny, f.bc, x, y, geo.data(), msg);
  if (st != SIDP_OK) return fail(c, st, msg);
  if (!c->d_geo && cudaMalloc(&c->d_geo, (size_t)kGeoFields * c->N * c->esize) != cudaSuccess)
    return fail(c, SIDP_ERR_OOM, "geometry allocation failed");
  if (!c->d_mass && cudaMalloc(&c->d_mass, (size_t)c->N * sizeof(double)) != cudaSuccess)
    return fail(c, SIDP_ERR_OOM, "geometry allocation failed");
  const sidp_status su = c->mixed ? upload<float>(c, c->d_geo, geo.data(), (long long)kGeoFields * c->N)
                                  : upload<double>(c, c->d_geo, geo.data(), (long long)kGeoFields * c->N);
  if (su != SIDP_OK) return su;
  CUDA_TRY(c, cudaMemcpy(c->d_mass, geo.data() + (size_t)GEO_MASS_FIELD * c->N, c->N * sizeof(double),
                         cudaMemcpyHostToDevice));
  c->hx.assign(x, x + c->N);
  c->hy.assign(y, y + c->N);
  c->curved = true;
  c->tuned = false;  // curved meshes have their own candidates (node and line layouts)
  c->settle = false;
  c->tile = 0;
  drop_graph(c);
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_set_time(sidp_ctx* c, double t) {
  if (!c || !std::isfinite(t)) return fail(c, SIDP_ERR_ARG, "bad argument");
  k_set_time<<<1, 1, 0, c->stream>>>(c->d_scal, t);
  CUDA_TRY(c, cudaGetLastError());
  return SIDP_OK;
}

sidp_status sidp_device_state(sidp_ctx* c, void** dptr, int* dtype, long long* stride) {
  if (!c || !dptr) return fail(c, SIDP_ERR_ARG, "null argument");
  *dptr = c->d_u[0];
  if (dtype) *dtype = c->mixed ? 1 : 0;
  if (stride) *stride = c->N;
  return SIDP_OK;
}

sidp_status sidp_compute_dt(sidp_ctx* c, double* dt) {
  if (!c || !dt) return fail(c, SIDP_ERR_ARG, "null argument");
  CUDA_TRY(c, run_dt(c, false));
  CUDA_TRY(c, cudaMemcpyAsync(dt, c->d_scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return SIDP_OK;
}

sidp_status sidp_stage(sidp_ctx* c, int k, double dt) {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  if (k < 1 || k > 3) return fail(c, SIDP_ERR_ARG, "stage must be 1, 2 or 3");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(c, SIDP_ERR_ARG, "dt must be finite and >= 0");
  if (k != 1 && c->stage_done != k - 1) return fail(c, SIDP_ERR_STATE, "stages must run in the order 1, 2, 3");
  k_set_scalar<<<1, 1, 0, c->stream>>>(c->d_scal, dt, k == 1 ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, run_stage(c, k));
  c->stage_done = (k == 3) ? 0 : k;
  return SIDP_OK;
}

sidp_status sidp_step(sidp_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return fail(c, SIDP_ERR_ARG, "bad argument");
  if (c->stage_done != 0) return fail(c, SIDP_ERR_STATE, "an SSP-RK3 step is half done (stage 1 or 2 ran)");
  int done = 0;
  if (nsteps > 0 && !c->tuned) {
    drop_graph(c);
    CUDA_TRY(c, autotune(c));
  }
  if (nsteps > 0 && c->settle) {
    if (c->steps < c->settle_at && c->steps + nsteps > c->settle_at) {  // the second pass falls inside
      const int k1 = (int)(c->settle_at - c->steps);
      const sidp_status st = sidp_step(c, k1);
      return st != SIDP_OK ? st : sidp_step(c, nsteps - k1);
    }
    if (c->steps >= c->settle_at) {
      drop_graph(c);
      c->graph_warm = false;
      CUDA_TRY(c, autotune(c, true));
    }
  }
  if (!c->use_graph || !c->graph_warm) {
    // first step eagerly: sets kernel attributes outside any capture
    if (nsteps > 0) {
      CUDA_TRY(c, run_step(c));
      ++done;
      c->graph_warm = true;
    }
  }
  if (c->use_graph && done < nsteps && !c->graph) {
    cudaGraph_t g = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = run_step(c);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(c, SIDP_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph = nullptr; return fail(c, SIDP_ERR_CUDA, cudaGetErrorString(e)); }
  }
  for (; done < nsteps; ++done) {
    if (c->use_graph && c->graph) CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
    else CUDA_TRY(c, run_step(c));
  }
  c->steps += nsteps;
  return SIDP_OK;
}

sidp_status sidp_set_graph(sidp_ctx* c, int on) {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  c->use_graph = on != 0;
  return SIDP_OK;
}

sidp_status sidp_set_stats(sidp_ctx* c, int on) {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  if ((on != 0) != c->stats_on) drop_graph(c);
  c->stats_on = on != 0;
  return SIDP_OK;
}

sidp_status sidp_set_debug(sidp_ctx* c, int on) try {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  if (on && !c->d_dbg) {
    if (cudaMalloc(&c->d_dbg, 4 * c->N * sizeof(double)) != cudaSuccess) return fail(c, SIDP_ERR_OOM, "debug allocation failed");
    CUDA_TRY(c, cudaMemset(c->d_dbg, 0, 4 * c->N * sizeof(double)));
  }
  if ((on != 0) != c->debug) drop_graph(c);
  c->debug = on != 0;
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_get_bounds(sidp_ctx* c, double* lo, double* hi, double* K, double* alpha) try {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  if (!c->d_dbg) return fail(c, SIDP_ERR_STATE, "debug capture was never enabled");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double* dst[4] = {lo, hi, K, alpha};
  for (int i = 0; i < 4; ++i)
    if (dst[i]) CUDA_TRY(c, cudaMemcpy(dst[i], c->d_dbg + i * c->N, c->N * sizeof(double), cudaMemcpyDeviceToHost));
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return fail(c, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(c, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_get_diag(sidp_ctx* c, sidp_diag* out) {
  if (!c || !out) return fail(c, SIDP_ERR_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  const int euler = c->cfg.law == SIDP_LAW_EULER2D;
  if (c->mixed)
    k_diag_partial<float><<<kDiagBlocks, 256, 0, c->stream>>>(static_cast<const float*>(c->d_u[0]), c->N, c->nc, c->n, c->h, c->d_wtab, c->cfg.gamma, euler, c->d_mass, c->d_part);
  else
    k_diag_partial<double><<<kDiagBlocks, 256, 0, c->stream>>>(static_cast<const double*>(c->d_u[0]), c->N, c->nc, c->n, c->h, c->d_wtab, c->cfg.gamma, euler, c->d_mass, c->d_part);
  CUDA_TRY(c, cudaGetLastError());
  k_diag_final<<<1, 32, 0, c->stream>>>(c->d_part, kDiagBlocks, c->d_diag);
  CUDA_TRY(c, cudaGetLastError());
  double d[kDiagK], sc[2];
  StageStats ss;
  CUDA_TRY(c, cudaMemcpyAsync(d, c->d_diag, sizeof(d), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(sc, c->d_scal, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&ss, c->d_stats, sizeof(ss), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out->t = sc[1];
  out->last_dt = sc[0];
  out->steps = c->steps;
  for (int f = 0; f < 4; ++f) {
    out->mass[f] = f < c->nc ? d[f] : 0.0;
    out->umin[f] = f < c->nc ? d[4 + f] : 0.0;
    out->umax[f] = f < c->nc ? d[8 + f] : 0.0;
  }
  out->rho_min = euler ? d[12] : 0.0;
  out->p_min = euler ? d[13] : 0.0;
  out->nonfinite = (long long)d[14];
  double bv, ev;
  std::memcpy(&bv, &ss.max_bound_violation, sizeof(double));
  std::memcpy(&ev, &ss.max_entropy_violation, sizeof(double));
  out->max_bound_violation = bv;
  out->max_entropy_violation = ev;
  out->rootfind_max_iters = (int)ss.rootfind_max_iters;
  out->rootfind_cap_hits = (long long)ss.rootfind_cap_hits;
  out->bound_nudges = (long long)ss.bound_nudges;
  if (out->nonfinite) return fail(c, SIDP_ERR_NONFINITE, "state holds non-finite values");
  return SIDP_OK;
}

sidp_status sidp_get_tile(const sidp_ctx* c, int* tx, int* ty) {
  if (!c) return fail(nullptr, SIDP_ERR_ARG, "null context");
  if (tx) *tx = tile_shape(c->cfg.p, c->tile).tx;
  if (ty) *ty = tile_shape(c->cfg.p, c->tile).ty;
  return SIDP_OK;
}

sidp_status sidp_set_tile(sidp_ctx* c, int index) {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  if (index < 0 || index >= num_tile_candidates(c->cfg.law))
    return fail(c, SIDP_ERR_ARG, "tile index out of range for this law");
  if (index != 0 && (c->cfg.limiter != 2 || c->cfg.smoothness || c->cfg.unsparsified))
    return fail(c, SIDP_ERR_ARG, "only subcell limiting without the smoothness indicator has tile candidates");
  if (index != 0 && c->curved && (index != kNumTiles || c->cfg.law != LAW_EULER))
    return fail(c, SIDP_ERR_ARG, "a curved mesh has two candidates: 0 (node layout) and 4 (line layout, Euler)");
  if (c->stage_done != 0) return fail(c, SIDP_ERR_STATE, "an SSP-RK3 step is half done (stage 1 or 2 ran)");
  c->tile = index;
  c->tuned = true;
  c->settle = false;
  drop_graph(c);
  return SIDP_OK;
}

sidp_status sidp_get_tile_index(const sidp_ctx* c, int* index) {
  if (!c || !index) return fail(nullptr, SIDP_ERR_ARG, "null argument");
  *index = c->tile;
  return SIDP_OK;
}

sidp_status sidp_synchronize(sidp_ctx* c) {
  if (!c) return fail(c, SIDP_ERR_ARG, "null context");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return SIDP_OK;
}

}  // extern "C"
