// Batched execution of independent problems (sidp_batch_*).
//
// Every instance owns a slice of three shared state buffers (u^n, u^(1), u^(2); each slice is the
// instance's [nc][N_i] field-major state in library node order) and its own time step.  Work is
// a task table of (instance, element tile) entries grouped by polynomial degree: each degree
// group is one launch of the tile kernel templated on that degree, over all tiles of all its
// instances.  A step is
//     dt launches (one per degree group) -> per-instance finalisation -> 3 x stage launches per group
// and is captured once in a CUDA graph that later steps replay.
//
// Instances moved onto curved meshes (sidp_batch_set_geometry) form degree groups of their own,
// launched with the curved-mesh kernels over tasks of (instance, block of EPB elements).
//
// Trade-off: one launch per degree group (the groups on concurrent graph branches) rather than
// one launch that switches on p inside.  Both exist: SIDP_BATCH_LAUNCH=single selects the single
// degree-switching launch (k_batch_all: default tile shapes, tasks by decreasing degree, the
// shared memory of the largest degree for every CTA, more register spills); on the 512-instance
// benchmark mix it measured 15.7 against 16.5 G node-updates/s for the groups, which stay the
// default.
#include <cfloat>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sidp.h"
#include "sidp_internal.h"

using namespace sidp;

namespace {

__global__ void k_batch_finalize(unsigned long long* bits, const double* cfl, double* dt, float* dtf, double* clock,
                                 int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double mn = __longlong_as_double((long long)bits[i]);
  const double v = (mn < DBL_MAX) ? cfl[i] * mn : 0.0;
  dt[i] = v;
  dtf[i] = (float)v;
  clock[i] += v;
  bits[i] = (unsigned long long)__double_as_longlong(DBL_MAX);
}

struct Group {
  int p = 0;  // degree and tile shape shared by the group's tasks
  bool curved = false;  // curved-mesh instances: tasks are (instance, element block), one shape
  int tile = 0;
  int2* d_tasks = nullptr;
  int ntasks = 0;
  // the group's task tables for every tile shape (subcell limiting without the smoothness
  // indicator: the batch autotuner chooses among them at the first step)
  int2* d_tasks_t[kMaxCand] = {};
  int ntasks_t[kMaxCand] = {};
};

thread_local std::string g_batch_err;

}  // namespace

struct sidp_batch {
  std::vector<sidp_config> cfgs;
  int n = 0, law = 0, nc = 1, limiter = 2;
  bool mixed = false;
  size_t esize = 8;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<long long> N, off;  // nodes and value offset of each instance
  // curved meshes (sidp_batch_set_geometry): per instance the device metric arrays (null while the
  // instance is Cartesian) and host copies of its node coordinates and masses
  std::vector<void*> d_geo;
  std::vector<std::vector<double>> hx, hy, hmass;
  bool any_shape = false;  // the groups keep task tables for every tile shape
  long long total_vals = 0;
  void* d_u[3] = {nullptr, nullptr, nullptr};
  void* d_inst[4] = {nullptr, nullptr, nullptr, nullptr};  // instance tables: dt, stage 1, 2, 3
  double* d_dt = nullptr;
  float* d_dtf = nullptr;
  double* d_clock = nullptr;
  double* d_cfl = nullptr;
  unsigned long long* d_bits = nullptr;
  StageStats* d_stats = nullptr;
  double* d_dbg = nullptr;  // debug capture: lo, hi, K, alpha-tilde, each [total nodes] (or null)
  bool debug = false;
  long long total_nodes = 0;
  std::vector<Group> groups;
  bool tuned = false;  // the per-group tile shapes have been chosen (or fixed)
  // single-launch mode (subcell limiting without the smoothness indicator, statistics off): one
  // launch per stage over the tiles of every degree, default tile shapes, tasks by decreasing degree
  bool single = false;
  int4* d_all_tasks = nullptr;
  int n_all_tasks = 0;
  void* d_tabs = nullptr;  // Tables<T>[kMaxP + 1]
  std::vector<cudaStream_t> gstream;  // one stream per degree group (the groups are independent)
  std::vector<cudaEvent_t> gdone;     // a group's work on its stream is done
  cudaEvent_t fork = nullptr;         // work so far on the batch stream is done
  cudaGraphExec_t graph = nullptr;
  bool warm = false;
  bool stats_on = true;
  long long steps = 0;
  std::string err;
};

namespace {

sidp_status bfail(sidp_batch* b, sidp_status s, const std::string& m) {
  if (b) b->err = m;
  g_batch_err = m;
  return s;
}

#define BCUDA(b, expr)                                                                               \
  do {                                                                                               \
    cudaError_t _e = (expr);                                                                         \
    if (_e != cudaSuccess) return bfail(b, SIDP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

template <typename T>
cudaError_t build_tables(sidp_batch* b) {
  std::vector<Instance<T>> tab[4];
  for (int k = 0; k < 4; ++k) tab[k].resize(b->n);
  T* u[3] = {static_cast<T*>(b->d_u[0]), static_cast<T*>(b->d_u[1]), static_cast<T*>(b->d_u[2])};
  const T* dtT;
  if constexpr (sizeof(T) == 4) dtT = reinterpret_cast<const T*>(b->d_dtf);
  else dtT = reinterpret_cast<const T*>(b->d_dt);
  for (int i = 0; i < b->n; ++i) {
    const sidp_config& c = b->cfgs[i];
    Instance<T> I;
    std::memset(&I, 0, sizeof(I));
    I.N = b->N[i];
    I.nx = c.nx;
    I.ny = c.ny;
    for (int s = 0; s < 4; ++s) I.bc[s] = c.bc[s];
    I.h = (c.x1 - c.x0) / c.nx;
    I.hT = T(I.h);
    I.x0 = T(c.x0);
    I.y0 = T(c.y0);
    I.dt = b->d_dt + i;
    I.dtT = dtT + i;
    I.stats = b->stats_on ? b->d_stats + i : nullptr;
    I.geo = static_cast<const T*>(b->d_geo[i]);
    const long long o = b->off[i];
    if (b->debug && b->d_dbg) {  // per-node captures at the instance's node offset
      const long long no = o / b->nc;
      I.dbg_lo = b->d_dbg + no;
      I.dbg_hi = b->d_dbg + b->total_nodes + no;
      I.dbg_K = b->d_dbg + 2 * b->total_nodes + no;
      I.dbg_alpha = b->d_dbg + 3 * b->total_nodes + no;
    }
    // dt launch reads u^n
    Instance<T> d = I;
    d.uin = u[0] + o;
    tab[0][i] = d;
    Instance<T> s1 = I;
    s1.uin = u[0] + o; s1.u0 = u[0] + o; s1.uout = u[1] + o; s1.c0 = T(0); s1.c1 = T(1);
    tab[1][i] = s1;
    Instance<T> s2 = I;
    s2.uin = u[1] + o; s2.u0 = u[0] + o; s2.uout = u[2] + o; s2.c0 = T(0.75); s2.c1 = T(0.25);
    tab[2][i] = s2;
    Instance<T> s3 = I;
    s3.uin = u[2] + o; s3.u0 = u[0] + o; s3.uout = u[0] + o; s3.c0 = T(1.0 / 3.0); s3.c1 = T(2.0 / 3.0);
    tab[3][i] = s3;
  }
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = cudaSuccess;
    if (!b->d_inst[k]) e = cudaMalloc(&b->d_inst[k], sizeof(Instance<T>) * b->n);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b->d_inst[k], tab[k].data(), sizeof(Instance<T>) * b->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int LAW, typename T>
cudaError_t launch_batch_law(int p, int tile, const BatchLaunch<T>& bl, bool dt, cudaStream_t s) {
  switch (p) {
    case 1: return launch_batch_p<LAW, T, 1>(tile, bl, dt, s);
    case 2: return launch_batch_p<LAW, T, 2>(tile, bl, dt, s);
    case 3: return launch_batch_p<LAW, T, 3>(tile, bl, dt, s);
    case 4: return launch_batch_p<LAW, T, 4>(tile, bl, dt, s);
    case 5: return launch_batch_p<LAW, T, 5>(tile, bl, dt, s);
    case 6: return launch_batch_p<LAW, T, 6>(tile, bl, dt, s);
    case 7: return launch_batch_p<LAW, T, 7>(tile, bl, dt, s);
    default: return cudaErrorInvalidValue;
  }
}

// k = 0: time-step launch; k = 1..3: SSP-RK3 stage k (Sec. 5), for degree group gi on stream st.
// timed: the timed stage kernels whatever the statistics switch (the batch autotuner).
template <typename T>
cudaError_t launch_group(sidp_batch* b, int gi, int k, cudaStream_t st, bool timed = false) {
  {
    const Group& gr = b->groups[gi];
    // the general stage kernels and the node kernel's statistics variant exist in the default shape
    // only: their launches take the group's default-shape task table; the line kernel has its own
    // statistics variant; the time step runs the node-kernel machinery (default shape with a line
    // tile)
    const bool line = gr.tile >= kNumTiles;
    const bool default_shape = (k > 0 && (b->limiter != 2 || b->cfgs[0].smoothness ||
                                          (b->stats_on && !timed && !line))) ||
                               (k == 0 && line);
    BatchLaunch<T> bl;
    std::memset(&bl, 0, sizeof(bl));
    bl.insts = static_cast<const Instance<T>*>(b->d_inst[k]);
    bl.tasks = default_shape ? gr.d_tasks_t[0] : gr.d_tasks;
    bl.ntasks = default_shape ? gr.ntasks_t[0] : gr.ntasks;
    double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
    gll_tables(gr.p, xi, w, D);
    const int nn = gr.p + 1;
    for (int i = 0; i < nn; ++i) { bl.tab.w[i] = T(w[i]); bl.tab.xi[i] = T(xi[i]); }
    for (int i = 0; i < nn * nn; ++i) bl.tab.D[i] = T(D[i]);
    bl.lp = make_law_params<T>(b->cfgs[0].gamma, b->cfgs[0].adv_beta, b->cfgs[0].adv_grad);
    {
      double Vinv[kMaxN * kMaxN], nrm[kMaxN];
      modal_tables(gr.p, Vinv, nrm);
      for (int i = 0; i < nn * nn; ++i) bl.tab.Vinv[i] = T(Vinv[i]);
      for (int i = 0; i < nn; ++i) bl.tab.nrm[i] = T(nrm[i]);
      sidp_config cp = b->cfgs[0];
      cp.p = gr.p;  // s0 defaults per degree
      bl.si = make_smoothness<T>(cp);
    }
    bl.limiter = b->limiter;
    bl.bits = b->d_bits;
    bl.stats = (b->stats_on && !timed) ? 1 : 0;
    bl.curved = gr.curved ? 1 : 0;
    const int tile = default_shape ? 0 : gr.tile;
    switch (b->law) {
      case LAW_BURGERS: return launch_batch_law<LAW_BURGERS, T>(gr.p, tile, bl, k == 0, st);
      case LAW_EULER: return launch_batch_law<LAW_EULER, T>(gr.p, tile, bl, k == 0, st);
      case LAW_ADVECTION_VAR: return launch_batch_law<LAW_ADVECTION_VAR, T>(gr.p, tile, bl, k == 0, st);
      default: return launch_batch_law<LAW_ADVECTION, T>(gr.p, tile, bl, k == 0, st);
    }
  }
}

template <typename T>
cudaError_t launch_all(sidp_batch* b, int k) {
  BatchAllLaunch<T> bl;
  std::memset(&bl, 0, sizeof(bl));
  bl.insts = static_cast<const Instance<T>*>(b->d_inst[k]);
  bl.tasks = b->d_all_tasks;
  bl.ntasks = b->n_all_tasks;
  bl.tabs = static_cast<const Tables<T>*>(b->d_tabs);
  bl.lp = make_law_params<T>(b->cfgs[0].gamma, b->cfgs[0].adv_beta, b->cfgs[0].adv_grad);
  bl.bits = b->d_bits;
  switch (b->law) {
    case LAW_BURGERS: return launch_batch_all<LAW_BURGERS, T>(bl, k == 0, b->stream);
    case LAW_EULER: return launch_batch_all<LAW_EULER, T>(bl, k == 0, b->stream);
    case LAW_ADVECTION_VAR: return launch_batch_all<LAW_ADVECTION_VAR, T>(bl, k == 0, b->stream);
    default: return launch_batch_all<LAW_ADVECTION, T>(bl, k == 0, b->stream);
  }
}

template <typename T>
cudaError_t upload_tables(sidp_batch* b) {
  std::vector<Tables<T>> tabs(kMaxP + 1);
  std::memset(tabs.data(), 0, tabs.size() * sizeof(Tables<T>));
  for (int p = 1; p <= kMaxP; ++p) {
    double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN], Vinv[kMaxN * kMaxN], nrm[kMaxN];
    gll_tables(p, xi, w, D);
    modal_tables(p, Vinv, nrm);
    const int nn = p + 1;
    for (int i = 0; i < nn; ++i) { tabs[p].w[i] = T(w[i]); tabs[p].xi[i] = T(xi[i]); tabs[p].nrm[i] = T(nrm[i]); }
    for (int i = 0; i < nn * nn; ++i) { tabs[p].D[i] = T(D[i]); tabs[p].Vinv[i] = T(Vinv[i]); }
  }
  cudaError_t e = cudaMalloc(&b->d_tabs, tabs.size() * sizeof(Tables<T>));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(b->d_tabs, tabs.data(), tabs.size() * sizeof(Tables<T>), cudaMemcpyHostToDevice);
}

// Launches k0..k1 of every degree group, each group on its own stream forked from the batch stream
// and joined back into it (under stream capture: parallel graph branches), so that one group's
// launch tail overlaps the others' work.
cudaError_t run_groups(sidp_batch* b, int k0, int k1) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    const cudaStream_t st = b->gstream[gi];
    e = cudaStreamWaitEvent(st, b->fork, 0);
    for (int k = k0; k <= k1 && e == cudaSuccess; ++k)
      e = b->mixed ? launch_group<float>(b, (int)gi, k, st) : launch_group<double>(b, (int)gi, k, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->gdone[gi], st);
  }
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) e = cudaStreamWaitEvent(b->stream, b->gdone[gi], 0);
  return e;
}

// One SSP-RK3 step of every instance: per-instance time steps (all groups), their finalize, then
// the three stages (all groups).
cudaError_t run_batch_step(sidp_batch* b) {
  const bool single = b->single && !b->stats_on;
  cudaError_t e = single ? (b->mixed ? launch_all<float>(b, 0) : launch_all<double>(b, 0)) : run_groups(b, 0, 0);
  if (e != cudaSuccess) return e;
  k_batch_finalize<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_bits, b->d_cfl, b->d_dt, b->d_dtf, b->d_clock, b->n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!single) return run_groups(b, 1, 3);
  for (int k = 1; k <= 3 && e == cudaSuccess; ++k) e = b->mixed ? launch_all<float>(b, k) : launch_all<double>(b, k);
  return e;
}

// Degree groups and their task tables: Cartesian instances of degree p, (instance, tile) for every
// tile shape (one tile shape per degree, the starting point of the batch autotuner: the
// single-instance tuner's choice when it has run for this (law, p, precision), else the default;
// the stage kernels of other limiters, of the smoothness indicator and of the statistics exist
// for the default shape only, so every group keeps a task table for that shape); curved-mesh
// instances of degree p, (instance, block of EPB elements).  A regrouping keeps the tile shape a
// Cartesian degree had.  One stream and one event per group.
cudaError_t build_groups(sidp_batch* b) {
  std::map<int, int> keep;
  for (Group& g : b->groups) {
    if (!g.curved) keep[g.p] = g.tile;
    for (int t = 0; t < kMaxCand; ++t) cudaFree(g.d_tasks_t[t]);
  }
  b->groups.clear();
  std::map<std::pair<int, int>, std::vector<int2>> tasks[kMaxCand];  // per tile shape: (curved, p) -> tasks
  for (int i = 0; i < b->n; ++i) {
    const sidp_config& c = b->cfgs[i];
    if (b->d_geo[i]) {
      const int nn = (c.p + 1) * (c.p + 1), epb = (256 / nn) > 0 ? 256 / nn : 1;  // CurvedGeom<p>::EPB
      const long long nb = ((long long)c.nx * c.ny + epb - 1) / epb;
      for (long long k = 0; k < nb; ++k) tasks[0][{1, c.p}].push_back(make_int2(i, (int)k));
      continue;
    }
    for (int tile = 0; tile < (b->any_shape ? num_tile_candidates(b->law) : 1); ++tile) {
      const TileShape ts = tile_shape(c.p, tile);
      const long long ntiles = (long long)((c.nx + ts.tx - 1) / ts.tx) * ((c.ny + ts.ty - 1) / ts.ty);
      for (long long t = 0; t < ntiles; ++t) tasks[tile][{0, c.p}].push_back(make_int2(i, (int)t));
    }
  }
  cudaError_t e = cudaSuccess;
  for (auto& kv : tasks[0]) {
    Group g;
    g.curved = kv.first.first != 0;
    g.p = kv.first.second;
    b->groups.push_back(g);
    Group& gr = b->groups.back();
    const int tables = (!gr.curved && b->any_shape) ? num_tile_candidates(b->law) : 1;
    for (int tile = 0; tile < tables; ++tile) {
      const std::vector<int2>& v = tasks[tile][kv.first];
      gr.ntasks_t[tile] = (int)v.size();
      if ((e = cudaMalloc(&gr.d_tasks_t[tile], sizeof(int2) * v.size())) != cudaSuccess) return e;
      if ((e = cudaMemcpy(gr.d_tasks_t[tile], v.data(), sizeof(int2) * v.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    }
    int tile = 0;
    if (!gr.curved && b->any_shape) {
      tile = keep.count(gr.p) ? keep[gr.p] : tuned_tile(b->law, gr.p, b->mixed ? 1 : 0);
      if (tile < 0) tile = 0;
    }
    gr.tile = tile;
    gr.d_tasks = gr.d_tasks_t[tile];
    gr.ntasks = gr.ntasks_t[tile];
  }
  while (b->gstream.size() < b->groups.size()) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    b->gstream.push_back(st);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    b->gdone.push_back(ev);
  }
  return cudaSuccess;
}

// Batch autotuner: with valid time steps in place (one time-step pass; the clocks are restored
// afterwards), time stage 1 of each degree group with each tile shape and keep the fastest.
// Stage 1 writes only u^(1), so the state is untouched.  The groups are tuned one after another
// on the batch stream.
cudaError_t tune_batch(sidp_batch* b) {
  std::vector<double> clock(b->n);
  cudaError_t e = cudaMemcpy(clock.data(), b->d_clock, b->n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  if ((e = run_groups(b, 0, 0)) != cudaSuccess) return e;
  k_batch_finalize<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_bits, b->d_cfl, b->d_dt, b->d_dtf, b->d_clock, b->n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    Group& g = b->groups[gi];
    if (g.curved) continue;  // one kernel shape on curved meshes
    float best = 1e30f;
    int best_t = g.tile;
    // the line kernel's tiles are candidates only for groups of large instances: on the meshes of
    // up to a few hundred thousand nodes that batches hold, its fewer and longer CTAs measured
    // slower over whole steps than the node kernel, although a lone stage 1 can time faster
    long long gn = 0, gc = 0;
    for (int i = 0; i < b->n; ++i)
      if (!b->d_geo[i] && b->cfgs[i].p == g.p) { gn += b->N[i]; ++gc; }
    const int ncand = (gc > 0 && gn / gc >= kLineMinNodes) ? num_tile_candidates(b->law) : kNumTiles;
    for (int t = 0; t < ncand && e == cudaSuccess; ++t) {
      g.tile = t;
      g.d_tasks = g.d_tasks_t[t];
      g.ntasks = g.ntasks_t[t];
      auto launch = [&]() {
        return b->mixed ? launch_group<float>(b, (int)gi, 1, b->stream, true)
                        : launch_group<double>(b, (int)gi, 1, b->stream, true);
      };
      if ((e = launch()) != cudaSuccess) break;  // warm-up (and kernel attributes)
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
      cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) { best = ms; best_t = t; }
    }
    g.tile = best_t;
    g.d_tasks = g.d_tasks_t[best_t];
    g.ntasks = g.ntasks_t[best_t];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_clock, clock.data(), b->n * sizeof(double), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

extern "C" {

sidp_status sidp_batch_create(sidp_batch** out, const sidp_config* cfgs, int count, void* cuda_stream) try {
  if (!out) return bfail(nullptr, SIDP_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (!cfgs || count < 1) return bfail(nullptr, SIDP_ERR_ARG, "empty batch");
  for (int i = 0; i < count; ++i) {
    std::string msg;
    if (validate_config(&cfgs[i], msg) != SIDP_OK) return bfail(nullptr, SIDP_ERR_ARG, "instance " + std::to_string(i) + ": " + msg);
    if (cfgs[i].law != cfgs[0].law || cfgs[i].precision != cfgs[0].precision || cfgs[i].limiter != cfgs[0].limiter ||
        cfgs[i].gamma != cfgs[0].gamma || cfgs[i].adv_beta[0] != cfgs[0].adv_beta[0] || cfgs[i].adv_beta[1] != cfgs[0].adv_beta[1] ||
        (cfgs[0].law == SIDP_LAW_ADVECTION_VAR2D &&
         (cfgs[i].adv_grad[0] != cfgs[0].adv_grad[0] || cfgs[i].adv_grad[1] != cfgs[0].adv_grad[1])) ||
        cfgs[i].smoothness != cfgs[0].smoothness || cfgs[i].si_s0 != cfgs[0].si_s0 || cfgs[i].si_kappa != cfgs[0].si_kappa ||
        cfgs[i].si_gmin != cfgs[0].si_gmin || cfgs[i].si_gmax != cfgs[0].si_gmax)
      return bfail(nullptr, SIDP_ERR_ARG, "all instances of a batch share law, precision, limiter, law and smoothness parameters");
    for (int s = 0; s < 4; ++s)
      if (cfgs[i].bc[s] == SIDP_BC_EXACT_STATE || cfgs[i].bc[s] == SIDP_BC_SPLIT)
        return bfail(nullptr, SIDP_ERR_ARG, "exact-state and split sides are not supported in batches");
    if (cfgs[i].unsparsified) return bfail(nullptr, SIDP_ERR_ARG, "the unsparsified comparison mode is not supported in batches");
  }
  sidp_batch* b = new sidp_batch();
  b->cfgs.assign(cfgs, cfgs + count);
  b->n = count;
  b->law = cfgs[0].law;
  b->nc = (b->law == SIDP_LAW_EULER2D) ? 4 : 1;
  b->limiter = cfgs[0].limiter;
  b->mixed = cfgs[0].precision == SIDP_MIXED;
  b->esize = b->mixed ? 4 : 8;
  auto bail = [&](sidp_status s, const std::string& m) {
    g_batch_err = m;
    sidp_batch_destroy(b);
    return s;
  };
  b->N.resize(count);
  b->off.resize(count);
  b->d_geo.assign(count, nullptr);
  b->hx.resize(count);
  b->hy.resize(count);
  b->hmass.resize(count);
  long long tot = 0;
  const bool any_shape = cfgs[0].limiter == 2 && !cfgs[0].smoothness;
  b->any_shape = any_shape;
  for (int i = 0; i < count; ++i) {
    const sidp_config& c = cfgs[i];
    const int nn = (c.p + 1) * (c.p + 1);
    b->N[i] = (long long)c.nx * c.ny * nn;
    b->off[i] = tot;
    tot += b->nc * b->N[i];
  }
  b->total_vals = tot;
  b->total_nodes = tot / b->nc;
  cudaError_t e;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
    b->own_stream = true;
  }
  for (int k = 0; k < 3; ++k)
    if (cudaMalloc(&b->d_u[k], tot * b->esize) != cudaSuccess) return bail(SIDP_ERR_OOM, "state allocation failed");
  if (cudaMalloc(&b->d_dt, count * sizeof(double)) != cudaSuccess || cudaMalloc(&b->d_dtf, count * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->d_clock, count * sizeof(double)) != cudaSuccess || cudaMalloc(&b->d_cfl, count * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->d_bits, count * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&b->d_stats, count * sizeof(StageStats)) != cudaSuccess)
    return bail(SIDP_ERR_OOM, "scratch allocation failed");
  std::vector<double> cfl(count), zero(count, 0.0);
  std::vector<unsigned long long> big(count, 0x7fefffffffffffffULL);
  std::vector<StageStats> zs(count);
  std::memset(zs.data(), 0, zs.size() * sizeof(StageStats));
  for (int i = 0; i < count; ++i) cfl[i] = cfgs[i].cfl;
  if ((e = cudaMemcpy(b->d_cfl, cfl.data(), count * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_clock, zero.data(), count * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_dt, zero.data(), count * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_bits, big.data(), count * sizeof(unsigned long long), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_stats, zs.data(), count * sizeof(StageStats), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->d_u[0], 0, tot * b->esize)) != cudaSuccess)
    return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  if ((e = b->mixed ? build_tables<float>(b) : build_tables<double>(b)) != cudaSuccess) return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  if ((e = build_groups(b)) != cudaSuccess) return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  // the batch autotuner runs at the first step unless a shape is forced or the table knows them
  b->tuned = !any_shape || std::getenv("SIDP_TILE") != nullptr ||
             (std::getenv("SIDP_AUTOTUNE") && std::getenv("SIDP_AUTOTUNE")[0] == '0');
  {  // SIDP_BATCH_LAUNCH=single: one launch per stage over every degree (measured slower than the
     // concurrent degree groups on the benchmark mix, so not the default)
    const char* mode = std::getenv("SIDP_BATCH_LAUNCH");
    b->single = any_shape && mode && std::string(mode) == "single";
  }
  if (b->single) {
    std::vector<int4> all;
    for (int p = kMaxP; p >= 1; --p)
      for (int i = 0; i < count; ++i) {
        if (cfgs[i].p != p) continue;
        const TileShape ts = kTiles[p][0];
        const long long ntiles = (long long)((cfgs[i].nx + ts.tx - 1) / ts.tx) * ((cfgs[i].ny + ts.ty - 1) / ts.ty);
        for (long long t = 0; t < ntiles; ++t) all.push_back(make_int4(i, (int)t, p, 0));
      }
    b->n_all_tasks = (int)all.size();
    if (cudaMalloc(&b->d_all_tasks, sizeof(int4) * all.size()) != cudaSuccess) return bail(SIDP_ERR_OOM, "task table allocation failed");
    if ((e = cudaMemcpy(b->d_all_tasks, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
    if ((e = b->mixed ? upload_tables<float>(b) : upload_tables<double>(b)) != cudaSuccess)
      return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  }
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return bail(SIDP_ERR_CUDA, cudaGetErrorString(e));
  *out = b;
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(nullptr, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(nullptr, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_destroy(sidp_batch* b) {
  if (!b) return SIDP_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (int k = 0; k < 3; ++k) cudaFree(b->d_u[k]);
  for (int k = 0; k < 4; ++k) cudaFree(b->d_inst[k]);
  for (auto& g : b->groups)
    for (int t = 0; t < kMaxCand; ++t) cudaFree(g.d_tasks_t[t]);
  cudaFree(b->d_all_tasks);
  cudaFree(b->d_tabs);
  cudaFree(b->d_dt);
  cudaFree(b->d_dtf);
  cudaFree(b->d_clock);
  cudaFree(b->d_cfl);
  cudaFree(b->d_bits);
  cudaFree(b->d_stats);
  cudaFree(b->d_dbg);
  for (void* gp : b->d_geo) cudaFree(gp);
  for (cudaStream_t st : b->gstream) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->gdone) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return SIDP_OK;
}

sidp_status sidp_batch_sizes(const sidp_batch* b, int i, long long* n_nodes, int* nc) {
  if (!b || i < 0 || i >= b->n) return bfail(nullptr, SIDP_ERR_ARG, "bad batch or index");
  if (n_nodes) *n_nodes = b->N[i];
  if (nc) *nc = b->nc;
  return SIDP_OK;
}

sidp_status sidp_batch_total_nodes(const sidp_batch* b, long long* n_nodes) {
  if (!b || !n_nodes) return bfail(nullptr, SIDP_ERR_ARG, "null argument");
  long long t = 0;
  for (long long v : b->N) t += v;
  *n_nodes = t;
  return SIDP_OK;
}

sidp_status sidp_batch_node_coords(const sidp_batch* b, int i, double* x, double* y) try {
  if (!b || i < 0 || i >= b->n || !x || !y) return bfail(nullptr, SIDP_ERR_ARG, "bad argument");
  if (b->d_geo[i]) {  // curved mesh: the coordinates it was given
    std::memcpy(x, b->hx[i].data(), b->N[i] * sizeof(double));
    std::memcpy(y, b->hy[i].data(), b->N[i] * sizeof(double));
    return SIDP_OK;
  }
  const sidp_config& c = b->cfgs[i];
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  gll_tables(c.p, xi, w, D);
  const int n = c.p + 1, NN = n * n;
  const double h = (c.x1 - c.x0) / c.nx;
  for (long long e = 0; e < (long long)c.nx * c.ny; ++e) {
    const long long ex = e % c.nx, ey = e / c.nx;
    for (int a = 0; a < n; ++a)
      for (int bb = 0; bb < n; ++bb) {
        x[e * NN + a * n + bb] = c.x0 + ((double)ex + xi[bb]) * h;
        y[e * NN + a * n + bb] = c.y0 + ((double)ey + xi[a]) * h;
      }
  }
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(nullptr, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(nullptr, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_set_geometry(sidp_batch* b, int i, const double* x, const double* y) try {
  if (!b || i < 0 || i >= b->n || !x || !y) return bfail(b, SIDP_ERR_ARG, "bad argument");
  const sidp_config& c = b->cfgs[i];
  if (c.law == SIDP_LAW_ADVECTION_VAR2D)
    return bfail(b, SIDP_ERR_ARG, "variable-velocity advection is defined on Cartesian meshes only");
  for (int k = 0; k < 4; ++k)
    if (c.bc[k] != SIDP_BC_PERIODIC && c.bc[k] != SIDP_BC_OUTFLOW && c.bc[k] != SIDP_BC_SLIP_WALL)
      return bfail(b, SIDP_ERR_ARG, "curved meshes take periodic, outflow or slip-wall sides");
  const long long N = b->N[i];
  std::vector<double> geo((size_t)kGeoFields * N);
  std::string msg;
  const sidp_status st = curved_metrics(c.p, c.nx, c.ny, c.bc, x, y, geo.data(), msg);
  if (st != SIDP_OK) return bfail(b, st, msg);
  BCUDA(b, cudaStreamSynchronize(b->stream));
  if (!b->d_geo[i] && cudaMalloc(&b->d_geo[i], (size_t)kGeoFields * N * b->esize) != cudaSuccess) {
    b->d_geo[i] = nullptr;
    return bfail(b, SIDP_ERR_OOM, "geometry allocation failed");
  }
  if (b->mixed) {
    std::vector<float> tmp(geo.begin(), geo.end());
    BCUDA(b, cudaMemcpy(b->d_geo[i], tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    BCUDA(b, cudaMemcpy(b->d_geo[i], geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  b->hx[i].assign(x, x + N);
  b->hy[i].assign(y, y + N);
  b->hmass[i].assign(geo.begin() + (size_t)GEO_MASS_FIELD * N, geo.begin() + (size_t)(GEO_MASS_FIELD + 1) * N);
  // regroup (the instance joins the curved group of its degree), new instance tables, a new graph;
  // the single-launch mode has no curved kernels
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  b->warm = false;
  b->single = false;
  BCUDA(b, b->mixed ? build_tables<float>(b) : build_tables<double>(b));
  BCUDA(b, build_groups(b));
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(b, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(b, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_set_state(sidp_batch* b, int i, const double* u) try {
  if (!b || i < 0 || i >= b->n || !u) return bfail(b, SIDP_ERR_ARG, "bad argument");
  const long long N = b->N[i], cnt = b->nc * N;
  for (long long j = 0; j < cnt; ++j)
    if (!std::isfinite(u[j])) return bfail(b, SIDP_ERR_NONFINITE, "state holds a non-finite value");
  if (b->law == SIDP_LAW_EULER2D) {
    const double g = b->cfgs[i].gamma;
    for (long long j = 0; j < N; ++j) {
      const double r = u[j], p = (g - 1.0) * (u[3 * N + j] - 0.5 * (u[N + j] * u[N + j] + u[2 * N + j] * u[2 * N + j]) / r);
      if (!(r > 0) || !(p > 0)) return bfail(b, SIDP_ERR_BOUNDS, "Euler state with rho <= 0 or p <= 0");
    }
  }
  double scale = 0.0;
  for (long long j = 0; j < N; ++j) scale = std::fmax(scale, std::fabs(u[j]));
  BCUDA(b, cudaMemcpy(reinterpret_cast<char*>(b->d_stats + i) + offsetof(StageStats, field_scale), &scale, sizeof(double),
                      cudaMemcpyHostToDevice));
  char* dst = static_cast<char*>(b->d_u[0]) + b->off[i] * b->esize;
  if (b->mixed) {
    std::vector<float> tmp(cnt);
    for (long long j = 0; j < cnt; ++j) tmp[j] = (float)u[j];
    BCUDA(b, cudaMemcpyAsync(dst, tmp.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
  } else {
    BCUDA(b, cudaMemcpyAsync(dst, u, cnt * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(b, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(b, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_get_buffer(sidp_batch* b, int i, int which, double* u) try {
  if (!b || i < 0 || i >= b->n || !u || which < 0 || which > 2) return bfail(b, SIDP_ERR_ARG, "bad argument");
  const long long cnt = b->nc * b->N[i];
  const char* src = static_cast<const char*>(b->d_u[which]) + b->off[i] * b->esize;
  if (b->mixed) {
    std::vector<float> tmp(cnt);
    BCUDA(b, cudaMemcpyAsync(tmp.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    for (long long j = 0; j < cnt; ++j) u[j] = tmp[j];
  } else {
    BCUDA(b, cudaMemcpyAsync(u, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(b, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(b, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_get_state(sidp_batch* b, int i, double* u) { return sidp_batch_get_buffer(b, i, 0, u); }

sidp_status sidp_batch_stage(sidp_batch* b, int k, const double* dt) try {
  if (!b || k < 1 || k > 3 || !dt) return bfail(b, SIDP_ERR_ARG, "bad argument");
  for (int i = 0; i < b->n; ++i)
    if (!(dt[i] >= 0.0) || !std::isfinite(dt[i])) return bfail(b, SIDP_ERR_ARG, "time steps must be finite and >= 0");
  std::vector<float> dtf(dt, dt + b->n);
  BCUDA(b, cudaStreamSynchronize(b->stream));
  BCUDA(b, cudaMemcpy(b->d_dt, dt, b->n * sizeof(double), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->d_dtf, dtf.data(), b->n * sizeof(float), cudaMemcpyHostToDevice));
  if (b->single && !b->stats_on) BCUDA(b, b->mixed ? launch_all<float>(b, k) : launch_all<double>(b, k));
  else BCUDA(b, run_groups(b, k, k));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(b, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(b, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_set_debug(sidp_batch* b, int on) {
  if (!b) return bfail(nullptr, SIDP_ERR_ARG, "null batch");
  if (on && !b->d_dbg) {
    if (cudaMalloc(&b->d_dbg, 4 * b->total_nodes * sizeof(double)) != cudaSuccess)
      return bfail(b, SIDP_ERR_OOM, "debug allocation failed");
    BCUDA(b, cudaMemset(b->d_dbg, 0, 4 * b->total_nodes * sizeof(double)));
  }
  if ((on != 0) == b->debug) return SIDP_OK;
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->debug = on != 0;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  BCUDA(b, b->mixed ? build_tables<float>(b) : build_tables<double>(b));
  return SIDP_OK;
}

sidp_status sidp_batch_get_bounds(sidp_batch* b, int i, double* lo, double* hi, double* K, double* alpha) {
  if (!b || i < 0 || i >= b->n) return bfail(b, SIDP_ERR_ARG, "bad argument");
  if (!b->d_dbg) return bfail(b, SIDP_ERR_STATE, "debug capture was never enabled");
  BCUDA(b, cudaStreamSynchronize(b->stream));
  double* dst[4] = {lo, hi, K, alpha};
  const long long no = b->off[i] / b->nc;
  for (int q = 0; q < 4; ++q)
    if (dst[q])
      BCUDA(b, cudaMemcpy(dst[q], b->d_dbg + q * b->total_nodes + no, b->N[i] * sizeof(double), cudaMemcpyDeviceToHost));
  return SIDP_OK;
}

sidp_status sidp_batch_step(sidp_batch* b, int nsteps) {
  if (!b || nsteps < 0) return bfail(b, SIDP_ERR_ARG, "bad argument");
  if (!b->tuned && nsteps > 0 && !(b->single && !b->stats_on)) {
    BCUDA(b, tune_batch(b));
    b->tuned = true;
  }
  int done = 0;
  if (!b->warm && nsteps > 0) {  // first step eagerly: kernel attributes are set outside capture
    BCUDA(b, run_batch_step(b));
    b->warm = true;
    ++done;
  }
  if (done < nsteps && !b->graph) {
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = run_batch_step(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, SIDP_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(b, SIDP_ERR_CUDA, cudaGetErrorString(e)); }
  }
  for (; done < nsteps; ++done) BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  b->steps += nsteps;
  return SIDP_OK;
}

sidp_status sidp_batch_get_diag(sidp_batch* b, int i, sidp_diag* out) try {
  if (!b || i < 0 || i >= b->n || !out) return bfail(b, SIDP_ERR_ARG, "bad argument");
  std::memset(out, 0, sizeof(*out));
  const sidp_config& c = b->cfgs[i];
  const long long N = b->N[i];
  std::vector<double> u(b->nc * N);
  sidp_status st = sidp_batch_get_state(b, i, u.data());
  if (st != SIDP_OK) return st;
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  gll_tables(c.p, xi, w, D);
  const int n = c.p + 1, NN = n * n;
  const double h = (c.x1 - c.x0) / c.nx;
  for (int f = 0; f < 4; ++f) { out->umin[f] = f < b->nc ? DBL_MAX : 0.0; out->umax[f] = f < b->nc ? -DBL_MAX : 0.0; }
  out->rho_min = out->p_min = (b->law == SIDP_LAW_EULER2D) ? DBL_MAX : 0.0;
  const bool curved = b->d_geo[i] != nullptr;
  for (long long j = 0; j < N; ++j) {
    const int node = (int)(j % NN);
    const double m = curved ? b->hmass[i][j] : h * h * w[node / n] * w[node % n];
    for (int f = 0; f < b->nc; ++f) {
      const double v = u[f * N + j];
      if (!std::isfinite(v)) { ++out->nonfinite; continue; }
      out->mass[f] += m * v;
      out->umin[f] = std::fmin(out->umin[f], v);
      out->umax[f] = std::fmax(out->umax[f], v);
    }
    if (b->law == SIDP_LAW_EULER2D) {
      const double r = u[j], p = (c.gamma - 1.0) * (u[3 * N + j] - 0.5 * (u[N + j] * u[N + j] + u[2 * N + j] * u[2 * N + j]) / r);
      out->rho_min = std::fmin(out->rho_min, r);
      out->p_min = std::fmin(out->p_min, p);
    }
  }
  StageStats ss;
  double sc[2];
  BCUDA(b, cudaMemcpy(&ss, b->d_stats + i, sizeof(ss), cudaMemcpyDeviceToHost));
  BCUDA(b, cudaMemcpy(&sc[0], b->d_clock + i, sizeof(double), cudaMemcpyDeviceToHost));
  BCUDA(b, cudaMemcpy(&sc[1], b->d_dt + i, sizeof(double), cudaMemcpyDeviceToHost));
  out->t = sc[0];
  out->last_dt = sc[1];
  out->steps = b->steps;
  std::memcpy(&out->max_bound_violation, &ss.max_bound_violation, sizeof(double));
  std::memcpy(&out->max_entropy_violation, &ss.max_entropy_violation, sizeof(double));
  out->rootfind_max_iters = (int)ss.rootfind_max_iters;
  out->rootfind_cap_hits = (long long)ss.rootfind_cap_hits;
  out->bound_nudges = (long long)ss.bound_nudges;
  if (out->nonfinite) return bfail(b, SIDP_ERR_NONFINITE, "state holds non-finite values");
  return SIDP_OK;
} catch (const std::bad_alloc&) {
  return bfail(b, SIDP_ERR_OOM, "host allocation failed");
} catch (...) {
  return bfail(b, SIDP_ERR_ARG, "unexpected host exception");
}

sidp_status sidp_batch_set_stats(sidp_batch* b, int on) {
  if (!b) return bfail(nullptr, SIDP_ERR_ARG, "null batch");
  if ((on != 0) == b->stats_on) return SIDP_OK;
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->stats_on = on != 0;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  BCUDA(b, b->mixed ? build_tables<float>(b) : build_tables<double>(b));
  return SIDP_OK;
}

sidp_status sidp_batch_synchronize(sidp_batch* b) {
  if (!b) return bfail(nullptr, SIDP_ERR_ARG, "null batch");
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return SIDP_OK;
}

const char* sidp_batch_last_error(const sidp_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
