// Fused stage kernel and CFL time-step kernel, templated on degree P, element tile TX x TY,
// law and precision T.
//
// A CTA owns a tile of TX x TY elements (an (TX n) x (TY n) grid of nodes, n = P + 1), one thread
// per node.  A stage is element-local once the face-neighbour traces are known, so the whole
// forward-Euler update (Sec. 4, Eq. subcell-fct / convex-fct) and the SSP-RK3 combination (Sec. 5)
// run in one kernel:
//   A  every node of the tile, plus the one-node halo around the tile, is loaded once; its
//      per-node quantities (velocity, pressure, sound speed, p^{-(g-1)/(2g)}, sigma) and fluxes
//      F_x, F_y go to shared memory.  Tile slots of elements outside a ragged mesh edge hold the
//      boundary ghost of the adjacent element, so faces need no special case.
//   B  every face of the node grid -- interior subcell faces and element faces alike -- is
//      evaluated once by a uniform loop over threads: lambda (Sec. 2.1.1), the face flux
//      1/2 (F_L + F_R) - lambda/2 (u_R - u_L) (the Lax-Friedrichs flux Eq. lax-friedrichs on
//      element faces; the sparsified operator Eq. didp with d_ij of Eq. dij on subcell faces),
//      and the bar state of the limited field (Eq. bar-states).
//   C  per node: r^H (strong form, Eq. ho-update: line contraction with D_1D plus the face
//      corrections), r^L (difference of face fluxes), u^L, the local bounds (Sec. 4.1.1 and 4.3)
//   D  subcell fluxes r-bar (prefix sums along element lines, Sec. 4.1.3) and alpha-tilde
//      (Zalesak on field 0; Euler: entropy line search over the gamma_d-scaled candidates)
//   E  alpha_{m,k} = min of the two adjacent alpha-tilde; limited update; RK combination.
// Each face flux is computed once and read by both adjacent nodes; faces on tile boundaries are
// computed by both tiles from identical (left, right) arguments.  Hence the update is
// conservative up to the rounding of the final sums.
#pragma once
#include <cfloat>
#include "sidp_internal.h"
#include "sidp_laws.cuh"

namespace sidp {

constexpr int kRootMaxIt = 60;

template <typename T> struct Prec;
// root_tol: bracket width at which the entropy line search stops.  entropy_margin: the float32
// path demands sigma >= K (1 + margin) so that evaluation error in float32 cannot leave the stored
// state below the bound: a few ulp of rho e (compensated, also where kinetic energy dominates),
// and the fast power rho^gamma = exp2(gamma log2 rho), whose relative error grows with
// |gamma log2 rho| (about 1.9e-6 at gamma = 1.4, |log2 rho| = 8) and enters both K_i and the
// candidates' psi_K: 4e-6 covers the two for densities from 1/256 to 256.
template <> struct Prec<double> { static constexpr double root_tol = 1e-13; static constexpr double entropy_margin = 0.0; };
template <> struct Prec<float> { static constexpr float root_tol = 2e-6f; static constexpr float entropy_margin = 4e-6f; };

template <typename T, int NC> struct alignas(NC == 4 ? 4 * sizeof(T) : NC == 2 ? 2 * sizeof(T) : sizeof(T)) Vec { T v[NC]; };



template <int P, int TX, int TY>
struct TileGeom {
  static constexpr int n = P + 1, NN = n * n, NE = TX * TY, NT = NE * NN;
  static constexpr int NX = TX * n, NY = TY * n;
  static constexpr int NH = 2 * NX + 2 * NY;  // halo slots: W[NY], E[NY], S[NX], N[NX]
  static constexpr int NS = NT + NH;
  static constexpr int hW = NT, hE = NT + NY, hS = NT + 2 * NY, hN = NT + 2 * NY + NX;
  // Faces, indexed by node slot so that a warp's face accesses fall in distinct shared-memory
  // banks like its node accesses: x face k < NT is the face on the left of node slot k, NT + row the
  // face on the tile's east edge; y face k < NT is the face below node slot k, NT + col the face on
  // the tile's north edge.
  static constexpr int NFX = NT + NY, NFY = NT + NX;
  static constexpr int THREADS = ((NT + 31) / 32) * 32;
  static constexpr int MINB = (THREADS <= 256) ? 4 : 2;  // register budget for 32 resident warps per SM
  __device__ __forceinline__ static int slot(int row, int col) {
    const int ty = row / n, a = row - ty * n, tx = col / n, b = col - tx * n;
    return (ty * TX + tx) * NN + a * n + b;
  }
  // the x face on the right of node slot t (b its x index in the element, at tile column col)
  __device__ __forceinline__ static int xface_right(int t, int b, int row, int col) {
    return (col == NX - 1) ? NT + row : t + ((b == P) ? NN - P : 1);
  }
  // the y face above node slot t (a its y index in the element, at tile row row)
  __device__ __forceinline__ static int yface_up(int t, int a, int row, int col) {
    return (row == NY - 1) ? NT + col : t + ((a == P) ? TX * NN - P * n : n);
  }
};

template <int P, int TX, int TY, class LAW, typename T>
struct TileSmem {
  using G = TileGeom<P, TX, TY>;
  using V = Vec<T, LAW::NC>;
  V u[G::NS];
  V fx[G::NS];  // F_x, later r_x on the node slots
  V fy[G::NS];  // F_y, later r_y
  V fbx[G::NFX];
  V fby[G::NFY];
  typename LAW::Aux aux[G::NS];
  T sig[LAW::kEntropy ? G::NS : 1];
  // per face: bar state of field 0 and, for Euler, min(sigma_L, sigma_R)
  Vec<T, LAW::kEntropy ? 2 : 1> bbx[G::NFX];
  Vec<T, LAW::kEntropy ? 2 : 1> bby[G::NFY];
  T alpha[G::NT];
  T D[G::NN];
  T w[G::n];
  T Vinv[G::NN];  // smoothness indicator: nodal -> modal transform
  T nrm[G::n];
  T eps[G::NE];   // smoothness factor epsilon_K per element of the tile
  T aK[G::NE];    // elementwise limiting: alpha_K per element of the tile
};

// The time-step kernel's shared memory: node states and records, one wave-speed bound per face,
// and the tables the tile loader fills.  About a third of TileSmem, so more CTAs fit on an SM.
template <int P, int TX, int TY, class LAW, typename T>
struct DtSmem {
  using G = TileGeom<P, TX, TY>;
  Vec<T, LAW::NC> u[G::NS];
  typename LAW::Aux aux[G::NS];
  T lamx[G::NFX];
  T lamy[G::NFY];
  T D[G::NN];
  T w[G::n];
  T Vinv[G::NN];
  T nrm[G::n];
};

// Ghost state of a split side (see SplitBC), decided in the stage precision (float64 in the FP64
// path; in float32 a node within rounding of the moving split point may take either state).
// own: the node's own trace.
template <int P, int NC, typename T>
__device__ __forceinline__ void split_ghost(const Instance<T>& I, int side, int ex, int ey, int pos, const T* xi,
                                            const T* own, T* out) {
  const SplitBC<T>& sp = I.split[side];
  const T c = (side < 2) ? I.y0 + I.hT * (T(ey) + xi[pos]) : I.x0 + I.hT * (T(ex) + xi[pos]);
  const T t = T(*I.tnow) + T(I.ck) * *I.dtT;
  if (c < T(sp.s0) + T(sp.speed) * t) {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = sp.a[f];
  } else if (!sp.wall_b) {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = sp.b[f];
  } else {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = own[f * I.N];
    if constexpr (NC == 4) out[side < 2 ? 1 : 2] = -out[side < 2 ? 1 : 2];
  }
}

// Trace of the neighbouring element across `side` (0 W, 1 E, 2 S, 3 N) of element (ex, ey) at
// position `pos` along the face.  Periodic wraps; outflow (reading: ghost = interior trace) copies
// the element's own trace node; exact-state reads the ghost buffer; a slip wall (Sec. 5.7) mirrors
// the own trace node (normal momentum negated); a split side takes one of two states (or the
// mirror) by the node's position against a moving split point.  xi: Gauss-Lobatto points on [0,1].
template <int P, int NC, typename T>
__device__ __forceinline__ void neighbor_trace(const Instance<T>& I, int side, int ex, int ey, int pos, const T* xi,
                                               T* out) {
  constexpr int n = P + 1, NN = n * n;
  const long long e = (long long)ey * I.nx + ex;
  long long ne = -1;
  int nd = 0, own = 0;
  const int bc = I.bc[side];
  switch (side) {
    case 0: nd = pos * n + P; own = pos * n; ne = (ex > 0) ? e - 1 : (bc == 0 ? e + (I.nx - 1) : -1); break;
    case 1: nd = pos * n; own = pos * n + P; ne = (ex < I.nx - 1) ? e + 1 : (bc == 0 ? e - (I.nx - 1) : -1); break;
    case 2: nd = P * n + pos; own = pos; ne = (ey > 0) ? e - I.nx : (bc == 0 ? e + (long long)(I.ny - 1) * I.nx : -1); break;
    default: nd = pos; own = P * n + pos; ne = (ey < I.ny - 1) ? e + I.nx : (bc == 0 ? e - (long long)(I.ny - 1) * I.nx : -1); break;
  }
  if (ne >= 0) {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = I.uin[f * I.N + ne * NN + nd];
  } else if (bc == 2 && I.ghost[side] != nullptr) {
    const long long nside = (side < 2) ? I.ny : I.nx;
    const long long along = (side < 2) ? ey : ex;
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = I.ghost[side][(f * nside + along) * n + pos];
  } else if (bc == 4 && I.split != nullptr && I.split[side].set) {
    split_ghost<P, NC>(I, side, ex, ey, pos, xi, I.uin + e * NN + own, out);
  } else {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = I.uin[f * I.N + e * NN + own];
    if constexpr (NC == 4) {  // slip wall (Euler): the mirror image, normal momentum negated
      if (bc == 3) out[side < 2 ? 1 : 2] = -out[side < 2 ? 1 : 2];
    }
  }
}

// Node quantities of a slot: state, aux and -- unless LEAN (time-step kernel) -- fluxes and sigma.
template <class L, class = void> struct HasPosition { static constexpr bool value = false; };
template <class L> struct HasPosition<L, decltype(void(L::kPosition))> { static constexpr bool value = L::kPosition; };

// The quantities of a thread's own node slot, kept in registers from phase A to phase B.
template <class LAW, typename T>
struct NodeRec {
  Vec<T, LAW::NC> u, fx, fy;
  typename LAW::Aux ax;
  T sig;
};

template <class LAW, bool LEAN, typename T, class S>
__device__ __forceinline__ void fill_slot(S& s, int slot, const T* uu, T x, T y, const LawParamsT<T>& lp,
                                          NodeRec<LAW, T>* rec = nullptr) {
  constexpr int NC = LAW::NC;
  typename LAW::Aux ax;
  if constexpr (HasPosition<LAW>::value) LAW::aux_at(uu, x, y, ax, lp);
  else LAW::aux(uu, ax, lp);
  Vec<T, NC> vu;
#pragma unroll
  for (int f = 0; f < NC; ++f) vu.v[f] = uu[f];
  s.u[slot] = vu;
  s.aux[slot] = ax;
  if constexpr (!LEAN) {
    Vec<T, NC> vx, vy;
    LAW::flux(uu, ax, 0, vx.v, lp);
    LAW::flux(uu, ax, 1, vy.v, lp);
    s.fx[slot] = vx;
    s.fy[slot] = vy;
    T sg = T(0);
    if constexpr (LAW::kEntropy) { sg = LAW::sigma(uu, ax, lp); s.sig[slot] = sg; }
    if (rec) { rec->u = vu; rec->fx = vx; rec->fy = vy; rec->ax = ax; rec->sig = sg; }
  }
}

// Phase A: node slots and the halo.  Returns true for threads that own an active mesh node.
// Halo slot h of a tile: the trace of the neighbouring element across the tile's edge (or the
// boundary ghost), and its position (the face node's; the normal velocity is continuous).
template <int P, int TX, int TY, int NC, typename T>
__device__ __forceinline__ void halo_load(const Instance<T>& I, const Tables<T>& tab, int h, int ex0, int ey0, T hh,
                                          T* uu, T& px, T& py) {
  using G = TileGeom<P, TX, TY>;
  constexpr int n = P + 1, NN = n * n;
  int side, pos;
  if (h < G::NY) { side = 0; pos = h; }
  else if (h < 2 * G::NY) { side = 1; pos = h - G::NY; }
  else if (h < 2 * G::NY + G::NX) { side = 2; pos = h - 2 * G::NY; }
  else { side = 3; pos = h - 2 * G::NY - G::NX; }
  int ex, ey, along;
  if (side < 2) { ex = (side == 0) ? ex0 : ex0 + TX - 1; ey = ey0 + pos / n; along = pos % n; }
  else { ey = (side == 2) ? ey0 : ey0 + TY - 1; ex = ex0 + pos / n; along = pos % n; }
  if (side < 2) {
    px = I.x0 + hh * T(side == 0 ? ex0 : ex0 + TX);
    py = I.y0 + hh * (T(ey) + tab.xi[along]);
  } else {
    px = I.x0 + hh * (T(ex) + tab.xi[along]);
    py = I.y0 + hh * T(side == 2 ? ey0 : ey0 + TY);
  }
  if (ex < I.nx && ey < I.ny) {
    neighbor_trace<P, NC>(I, side, ex, ey, along, tab.xi, uu);
  } else {
#pragma unroll
    for (int f = 0; f < NC; ++f) uu[f] = I.uin[f * I.N + ((long long)ey0 * I.nx + ex0) * NN];
  }
}

template <int P, int TX, int TY, class LAW, bool LEAN, typename T, class S>
__device__ __forceinline__ bool load_tile(S& s, const Instance<T>& I, const Tables<T>& tab, const LawParamsT<T>& lp,
                                          int tile_x, int tile_y, int& le, int& a, int& b, long long& g,
                                          NodeRec<LAW, T>* rec = nullptr) {
  using G = TileGeom<P, TX, TY>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const int t = threadIdx.x;
  const int ex0 = tile_x * TX, ey0 = tile_y * TY;
  if (t < NN) { s.D[t] = tab.D[t]; s.Vinv[t] = tab.Vinv[t]; }
  const T hh = I.hT;
  if (t < n) { s.w[t] = tab.w[t]; s.nrm[t] = tab.nrm[t]; }
  bool act = false;
  le = 0; a = 0; b = 0; g = 0;
  if (t < G::NT) {
    le = t / NN;
    const int node = t - le * NN;
    a = node / n;
    b = node - a * n;
    const int ex = ex0 + le % TX, ey = ey0 + le / TX;
    // node position (velocity laws); slots outside the mesh take the boundary face's position
    const T px = I.x0 + hh * (ex < I.nx ? T(ex) + tab.xi[b] : T(I.nx));
    const T py = I.y0 + hh * (ey < I.ny ? T(ey) + tab.xi[a] : T(I.ny));
    T uu[NC];
    if (ex < I.nx && ey < I.ny) {
      act = true;
      g = ((long long)ey * I.nx + ex) * NN + node;
#pragma unroll
      for (int f = 0; f < NC; ++f) uu[f] = I.uin[f * I.N + g];
    } else if (ey < I.ny) {
      neighbor_trace<P, NC>(I, 1, I.nx - 1, ey, a, tab.xi, uu);  // east of the mesh: ghost of the last element
    } else if (ex < I.nx) {
      neighbor_trace<P, NC>(I, 3, ex, I.ny - 1, b, tab.xi, uu);  // north of the mesh
    } else {
#pragma unroll
      for (int f = 0; f < NC; ++f) uu[f] = I.uin[f * I.N + ((long long)ey0 * I.nx + ex0) * NN];
    }
    // the thread's first halo slot is loaded before the node slot is processed, so that the two
    // global-load latencies overlap instead of adding up on the threads that own halo slots
    T uh[NC], hx = T(0), hy = T(0);
    if (t < G::NH) halo_load<P, TX, TY, NC>(I, tab, t, ex0, ey0, hh, uh, hx, hy);
    fill_slot<LAW, LEAN>(s, t, uu, px, py, lp, rec);
    if (t < G::NH) fill_slot<LAW, LEAN>(s, G::NT + t, uh, hx, hy, lp);
  }
  for (int h = (t < G::NT) ? t + G::THREADS : t; h < G::NH; h += G::THREADS) {
    T uu[NC], px, py;
    halo_load<P, TX, TY, NC>(I, tab, h, ex0, ey0, hh, uu, px, py);
    fill_slot<LAW, LEAN>(s, G::NT + h, uu, px, py, lp);
  }
  return act;
}

// Euler: largest t in [0, tcap] such that every candidate u^L + t w_c (w_c = gamma_d dt/m (+-r-bar))
// has rho > 0 and psi_K >= min(0, psi_K(u^L)).  psi_K is concave, so along each candidate the
// admissible set is an interval [0, t*]; candidates are processed in turn with the running cap.
// Root search: bracket [tL feasible, tR infeasible]; chord from the feasible end (stays feasible
// by concavity) and tangent from the infeasible end (stays infeasible), each classified by an
// actual evaluation, with a bisection step whenever the bracket did not halve.  Bounded by
// kRootMaxIt iterations (then the feasible end is returned and the cap is counted).
template <class LAW, typename T>
__device__ __forceinline__ void candidate(int c, const T* xp, const T* xm, const T* yp, const T* ym, T sc, T* w) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T v = (c == 0) ? xp[q] : (c == 1) ? -xm[q] : (c == 2) ? yp[q] : -ym[q];
    w[q] = sc * v;
  }
}

// Largest t in [0, tmax_] with u^L + t w admissible ({rho > 0, psi_K >= target}), given that t = 0 is
// and t = tmax_ is not.  psi_K is concave along the line, so the admissible t form [0, t*].  Bracket
// [tL feasible, tR infeasible]: chord from the feasible end (stays feasible by concavity), tangent
// from the infeasible end (stays infeasible), each classified by an actual evaluation, and a
// bisection step whenever the bracket did not halve.  At most kRootMaxIt iterations (the feasible
// end is returned and the cap counted).
template <class LAW, typename T>
__device__ T entropy_root(const T* uL, const T* w, T K, T psi0, T target, T tmax_, const LawParamsT<T>& lp,
                          int& iters, int& caps) {
  T tL = T(0), fL = psi0 - target, tR = tmax_;
  if (w[0] < T(0)) tR = tmin(tR, fdiv(-uL[0], w[0]));
  int it = 0;
#pragma unroll 1
  for (; it < kRootMaxIt; ++it) {
    const T width = tR - tL;
    if (!(width > Prec<T>::root_tol)) break;
    T uR[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) uR[f] = uL[f] + tR * w[f];
    if (uR[0] > T(0)) {
      const T fR = LAW::psi(uR, K, lp) - target;
      if (fR >= T(0)) { tL = tR; fL = fR; break; }
      const T tc = tL + fdiv(fL * (tR - tL), fL - fR);  // chord root: feasible side
      if (tc > tL && tc < tR) {
        T uc[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) uc[f] = uL[f] + tc * w[f];
        const T fc = (uc[0] > T(0)) ? LAW::psi(uc, K, lp) - target : T(-1);
        if (uc[0] > T(0) && fc >= T(0)) { tL = tc; fL = fc; } else { tR = tc; }
      }
      const T dR = LAW::psi_grad_dot(uR, K, w, lp);  // tangent root from the old tR: infeasible side
      if (dR < T(0)) {
        const T tn = tR - fdiv(fR, dR);
        if (tn > tL && tn < tR) {
          T un[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) un[f] = uL[f] + tn * w[f];
          const T fn = (un[0] > T(0)) ? LAW::psi(un, K, lp) - target : T(-1);
          if (un[0] > T(0) && fn >= T(0)) { tL = tn; fL = fn; } else { tR = tn; }
        }
      }
    }
    if (tR - tL > T(0.5) * width) {  // guarantee at least a halving
      const T tm = T(0.5) * (tL + tR);
      T um[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) um[f] = uL[f] + tm * w[f];
      const T fm = (um[0] > T(0)) ? LAW::psi(um, K, lp) - target : T(-1);
      if (um[0] > T(0) && fm >= T(0)) { tL = tm; fL = fm; } else { tR = tm; }
    }
  }
  if (it > iters) iters = it;
  if (it >= kRootMaxIt) ++caps;
  return tL;
}

// Euler: largest t in [0, tcap] such that every candidate u^L + t w_c, w_c = gamma_d dt/m (+-r-bar),
// has rho > 0 and psi_K >= min(0, psi_K(u^L)).  Along each candidate the admissible set is an
// interval [0, t*], so the candidates are taken in turn with the running cap.  First all four
// are tested at tcap against psi_K >= 0 (stricter than the target min(0, psi_K(u^L))) with the
// cheap certified test, without branches; only when some candidate is undecided are the target
// and the precise tests evaluated, and only those that fail there need a root search.
template <class LAW, typename T>
__device__ T entropy_limit(const T* uL, T K, const T* xp, const T* xm, const T* yp, const T* ym, T sc, T tcap,
                           const LawParamsT<T>& lp, int& iters, int& caps) {
  if (!(tcap > T(0))) return tcap;
  const T ts = tcap * sc;
  unsigned undecided = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T ut[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T v = (c == 0) ? xp[f] : (c == 1) ? -xm[f] : (c == 2) ? yp[f] : -ym[f];
      // float64 keeps the oracle's order of operations, u^L + t (scale r-bar)
      ut[f] = (sizeof(T) == 8) ? uL[f] + tcap * (sc * v) : uL[f] + ts * v;
    }
    const bool ok = (ut[0] > T(0)) && LAW::psi_certainly_ge(ut, K, T(0), lp);
    undecided |= ok ? 0u : (1u << c);
  }
  if (!undecided) return tcap;
  // target = min(0, psi_K(u^L)); the precise psi is needed only when u^L is not certainly inside
  const T target = LAW::psi_certainly_ge(uL, K, T(0), lp) ? T(0) : tmin(LAW::psi(uL, K, lp), T(0));
  unsigned fail = 0;
#pragma unroll 1
  while (undecided) {
    const int c = __ffs(undecided) - 1;
    undecided &= undecided - 1;
    T ut[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T v = (c == 0) ? xp[f] : (c == 1) ? -xm[f] : (c == 2) ? yp[f] : -ym[f];
      // float64 keeps the oracle's order of operations, u^L + t (scale r-bar)
      ut[f] = (sizeof(T) == 8) ? uL[f] + tcap * (sc * v) : uL[f] + ts * v;
    }
    // the precise psi only: the cheap certified test against target has just failed against 0
    // for this candidate, and target = min(0, psi_K(u^L)) lies within the test's error allowance
    // of 0 (u^L is in the entropy set up to rounding), so it cannot pass either
    if (!(ut[0] > T(0) && LAW::psi(ut, K, lp) >= target)) fail |= 1u << c;
  }
  if (!fail) return tcap;
  const T psi0 = LAW::psi(uL, K, lp);
  T t = tcap;
#pragma unroll 1
  while (fail) {
    const int c = __ffs(fail) - 1;
    fail &= fail - 1;
    T w[4];
    candidate<LAW>(c, xp, xm, yp, ym, sc, w);
    T ut[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) ut[f] = uL[f] + t * w[f];
    if (t < tcap && ut[0] > T(0) && LAW::psi(ut, K, lp) >= target) continue;  // admissible at the reduced cap
    t = entropy_root<LAW>(uL, w, K, psi0, target, t, lp, iters, caps);
    if (!(t > T(0))) break;
  }
  return t;
}

// True when every candidate u^L + tcap w_c is certainly admissible (rho > 0 and psi_K >= 0 by the
// cheap certified test, which implies psi_K >= min(0, psi_K(u^L))), or tcap <= 0: then
// entropy_limit returns tcap unchanged.  False: entropy_limit must be evaluated.
template <class LAW, typename T>
__device__ __forceinline__ bool entropy_certain(const T* uL, T K, const T* xp, const T* xm, const T* yp, const T* ym,
                                                T sc, T tcap, const LawParamsT<T>& lp) {
  if (!(tcap > T(0))) return true;
  const T ts = tcap * sc;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T ut[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T v = (c == 0) ? xp[f] : (c == 1) ? -xm[f] : (c == 2) ? yp[f] : -ym[f];
      ut[f] = (sizeof(T) == 8) ? uL[f] + tcap * (sc * v) : uL[f] + ts * v;
    }
    ok = ok && (ut[0] > T(0)) && LAW::psi_certainly_ge(ut, K, T(0), lp);
  }
  return ok;
}

// Post-round acceptance of the float32 store.  The limited field's forward-Euler result lies in
// its local bounds [lo, hi] in exact arithmetic (Sec. 4.1.3; Sec. 4.3 for the density); the
// float32 evaluation of the update can leave it outside by the rounding of its operands, of
// magnitude `mag` (the low-order state, the limited antidiffusive terms and the bounds).  A result
// outside by no more than 8 float32 ulp of `mag` is set onto the violated bound, so that the
// stored state satisfies the bounds exactly; the change is of the order of the update's own
// rounding, like the rounding of the store itself.  Returns 1 when the value moved.  The float64
// path keeps its result (no acceptance step: it is held to the float64 oracle).
template <typename T>
__device__ __forceinline__ int accept_rounded(T& v, T lo, T hi, T mag) {
  if constexpr (sizeof(T) == 8) {
    return 0;
  } else {
    const T tol = T(8) * FLT_EPSILON * mag;
    const bool below = (v < lo) && (v >= lo - tol), above = (v > hi) && (v <= hi + tol);
    v = below ? lo : (above ? hi : v);
    return (below || above) ? 1 : 0;
  }
}

template <typename T>
__device__ __forceinline__ void warp_max_atomic(T v, unsigned long long* dst) {
  double d = (double)v;  // v >= 0
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0 && d > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(d));
}

// Root-search counters of a warp: one atomic per warp (not per thread: on a flow with many
// limited nodes per-thread atomics on one address serialise).  All 32 lanes call it.
__device__ __forceinline__ void warp_rootfind_stats(int caps, int iters, int nudged, StageStats* st) {
  const unsigned c = __reduce_add_sync(0xffffffffu, (unsigned)caps);
  const unsigned m = __reduce_max_sync(0xffffffffu, (unsigned)iters);
  const unsigned g = __reduce_add_sync(0xffffffffu, (unsigned)nudged);
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(&st->rootfind_cap_hits, (unsigned long long)c);
    if (m) atomicMax(&st->rootfind_max_iters, m);
    if (g) atomicAdd(&st->bound_nudges, (unsigned long long)g);
  }
}

// Euler: largest t in [0, tcap] with u^L + t w in {rho > 0, psi_K >= min(0, psi_K(u^L))} for the
// single direction w (elementwise limiting, Eq. convex-provisional-elementwise).
template <class LAW, typename T>
__device__ T entropy_limit_dir(const T* uL, T K, const T* w, T tcap, const LawParamsT<T>& lp, int& iters, int& caps) {
  if (!(tcap > T(0))) return tcap;
  const T target = LAW::psi_certainly_ge(uL, K, T(0), lp) ? T(0) : tmin(LAW::psi(uL, K, lp), T(0));
  T ut[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) ut[f] = uL[f] + tcap * w[f];
  if (ut[0] > T(0) && (LAW::psi_certainly_ge(ut, K, target, lp) || LAW::psi(ut, K, lp) >= target)) return tcap;
  return entropy_root<LAW>(uL, w, K, LAW::psi(uL, K, lp), target, tcap, lp, iters, caps);
}

// Slots of the four neighbours of node slot t = (le, a, b) at tile position (row, col):
// within the element, across an element face inside the tile, or in the halo.
template <int P, int TX, int TY>
struct Nbr {
  using G = TileGeom<P, TX, TY>;
  static constexpr int n = P + 1, NN = n * n;
  __device__ __forceinline__ static int left(int t, int b, int row, int col) {
    return (col == 0) ? G::hW + row : t - ((b == 0) ? NN - P : 1);
  }
  __device__ __forceinline__ static int right(int t, int b, int row, int col) {
    return (col == G::NX - 1) ? G::hE + row : t + ((b == P) ? NN - P : 1);
  }
  __device__ __forceinline__ static int down(int t, int a, int row, int col) {
    return (row == 0) ? G::hS + col : t - ((a == 0) ? TX * NN - P * n : n);
  }
  __device__ __forceinline__ static int up(int t, int a, int row, int col) {
    return (row == G::NY - 1) ? G::hN + col : t + ((a == P) ? TX * NN - P * n : n);
  }
};

// Operand scale of the low-order state of node slot me (the limited field): |u_i| + 2 max_j |u_j|
// over its stencil (the four neighbours; with the unsparsified operator also every node of its
// two element lines).  u^L_i is u_i plus pair terms whose operands are bounded by
// lambda (|u_i| + |u_j|) (for the limited field |F.e| <= lambda |u|), and the CFL condition gives
// dt/m_i sum_j d_ij <= 1/2, so its float32 rounding is a few ulp of this scale.  Read from the
// stage input still in shared memory; called only for a result outside its bounds.
template <int P, int TX, int TY, bool DENSE, class S>
__device__ __forceinline__ auto stencil_scale(const S& s, int me, int le, int a, int b, int row, int col) {
  using N4 = Nbr<P, TX, TY>;
  constexpr int n = P + 1, NN = n * n;
  auto S0 = fabs(s.u[N4::left(me, b, row, col)].v[0]);
  S0 = tmax(S0, fabs(s.u[N4::right(me, b, row, col)].v[0]));
  S0 = tmax(S0, fabs(s.u[N4::down(me, a, row, col)].v[0]));
  S0 = tmax(S0, fabs(s.u[N4::up(me, a, row, col)].v[0]));
  if constexpr (DENSE) {
#pragma unroll 1
    for (int c = 0; c < n; ++c) S0 = tmax(S0, tmax(fabs(s.u[le * NN + a * n + c].v[0]), fabs(s.u[le * NN + c * n + b].v[0])));
  }
  return fabs(s.u[me].v[0]) + decltype(S0)(2) * S0;
}

// Entropy-bound violation of a limited result fe at node slot me: max(0, 1 - sigma(fe) / K_i) with
// K_i = min sigma over the node and its four neighbours of the stage input (still in shared
// memory).  sigma is evaluated accurately - compensated rho e (a few ulp even where kinetic energy
// dominates) and the correctly rounding-class powf (not the fast intrinsic), the ratio in
// float64 - so that the statistic measures the result against the bound of its input to a few
// 1e-7, not the ~1e-6 rounding of the limiter's fast float32 evaluation.  Statistics only.
template <int P, int TX, int TY, class LAW, typename T, class S>
__device__ __forceinline__ double entropy_violation64(const S& s, int me, int a, int b, int row, int col, const T* fe,
                                                      const LawParamsT<T>& lp) {
  auto sig = [&](const T* u) { return (double)LAW::rhoe(u) * (double)powf(u[0], -lp.gamma); };
  using N4 = Nbr<P, TX, TY>;
  double K = sig(s.u[me].v);
  K = fmin(K, sig(s.u[N4::left(me, b, row, col)].v));
  K = fmin(K, sig(s.u[N4::right(me, b, row, col)].v));
  K = fmin(K, sig(s.u[N4::down(me, a, row, col)].v));
  K = fmin(K, sig(s.u[N4::up(me, a, row, col)].v));
  if (!((double)fe[0] > 0.0)) return 1.0;
  return fmax(0.0, 1.0 - sig(fe) / K);
}

// Stage statistics of one node (all lanes of the warp call it): the limited field's excess over its
// local bounds relative to max(|bound|, field scale), the entropy-bound violation (float64 measure on
// the float32 path), and the root-search counters; warp-reduced, one atomic per warp and quantity.
template <int P, int TX, int TY, class LAW, typename T, bool DENSE, class S>
__device__ __forceinline__ void stage_stats(const S& s, const Instance<T>& I, const LawParamsT<T>& lp, bool on,
                                         Vec<T, LAW::NC> fe, T lo, T hi, T K, int caps, int iters, int nudged, int me,
                                         int a, int b, int row, int col) {
  T v = T(0), ev = T(0);
  if (on) {
    // relative to the local bound, floored at the field's magnitude (bounds that are zero up to
    // rounding would otherwise turn rounding into large relative values)
    const T scale = tmax(tmax(fabs(lo), fabs(hi)), T(I.stats->field_scale));
    v = tmax(lo - fe.v[0], fe.v[0] - hi);
    v = (v > T(0)) ? fdiv(v, scale > T(0) ? scale : T(1)) : T(0);
    if constexpr (LAW::kEntropy) {
      if constexpr (sizeof(T) == 4 && !DENSE) {
        ev = T(entropy_violation64<P, TX, TY, LAW, T>(s, me, a, b, row, col, fe.v, lp));
      } else {
        const T sg = LAW::sigma_of(fe.v, lp);
        ev = tmax(T(0), T(1) - sg / K);
        if (!(fe.v[0] > T(0))) ev = T(1);
      }
    }
  }
  warp_rootfind_stats(caps, iters, nudged, I.stats);
  warp_max_atomic(v, &I.stats->max_bound_violation);
  warp_max_atomic(ev, &I.stats->max_entropy_violation);
}

// Elementwise limiting (Sec. 4.1.2 linear, Sec. 4.2.1 convex constraints): alpha-tilde_i is the
// largest coefficient in [0,1] keeping u^L_i + alpha (dt/m_i) r_i, r_i = sum_k (r^H_ik - r^L_ik),
// inside the bounds of the limited field (Zalesak with the single flux r_i) and, for Euler, in
// the entropy set; every node of element K then takes alpha_K = min over K.  Writes u^FE with
// the SSP-RK3 combination and the stage statistics.
template <int P, int TX, int TY, class LAW, typename T, bool DENSE, class S>
__device__ __forceinline__ void elementwise_update(S& s, const Instance<T>& I, const LawParamsT<T>& lp, bool slot, bool act,
                                                bool move, long long g, int le, int me, int a, int b, const T* uL,
                                                const T* rx, const T* ry, T lo, T hi, T K, T m, T dt, T dtm) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const long long N = I.N;
  T rn[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) rn[q] = rx[q] + ry[q];
  T at = T(1);
  int iters = 0, caps = 0;
  if (slot) {
    if (move) {
      const T mdt = fdiv(m, dt);
      const T Qp = tmax(T(0), mdt * (hi - uL[0]));
      const T Qm = tmin(T(0), mdt * (lo - uL[0]));
      const T Rp = (rn[0] > T(0)) ? tmin(T(1), fdiv(Qp, rn[0])) : T(1);
      const T Rm = (rn[0] < T(0)) ? tmin(T(1), fdiv(Qm, rn[0])) : T(1);
      at = tmin(Rp, Rm);
      if constexpr (LAW::kEntropy) {
        T w[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) w[q] = dtm * rn[q];
        at = entropy_limit_dir<LAW>(uL, K * (T(1) + Prec<T>::entropy_margin), w, at, lp, iters, caps);
      }
    }
    s.alpha[me] = at;
    if (I.dbg_lo && act) {
      I.dbg_lo[g] = (double)lo;
      I.dbg_hi[g] = (double)hi;
      I.dbg_K[g] = (double)K;
      I.dbg_alpha[g] = (double)at;
    }
  }
  __syncthreads();
  if (slot && a == 0 && b == 0) {
    T mn = T(1);
    for (int i = 0; i < NN; ++i) mn = tmin(mn, s.alpha[le * NN + i]);
    s.aK[le] = mn;
  }
  __syncthreads();
  T fe[NC];
  int nudged = 0;
  if (slot) {
    const T ak = s.aK[le];
#pragma unroll
    for (int q = 0; q < NC; ++q) fe[q] = uL[q] + ak * dtm * rn[q];
    if constexpr (sizeof(T) == 4) {
      if (!(fe[0] >= lo && fe[0] <= hi)) {  // rare: the rounding scale only where it is needed
        const int row = (le / TX) * n + a, col = (le % TX) * n + b;
        nudged = accept_rounded(fe[0], lo, hi, stencil_scale<P, TX, TY, DENSE>(s, me, le, a, b, row, col) +
                                                   fabs(uL[0]) + fabs(ak * dtm * rn[0]) + tmax(fabs(lo), fabs(hi)));
      }
    }
    if (act) {
#pragma unroll
      for (int q = 0; q < NC; ++q)
        I.uout[q * N + g] = (I.c0 == T(0)) ? fe[q] : I.c0 * I.u0[q * N + g] + I.c1 * fe[q];
    }
  }
  if (I.stats) {  // statistics, out of line
    Vec<T, NC> vf;
#pragma unroll
    for (int q = 0; q < NC; ++q) vf.v[q] = fe[q];
    stage_stats<P, TX, TY, LAW, T, DENSE>(s, I, lp, act && move, vf, lo, hi, K, caps, iters, act ? nudged : 0, me,
                                          a, b, (le / TX) * n + a, (le % TX) * n + b);
  }
}

// Face along +e_k between the left/lower slot L (read from shared memory) and a right/upper state
// given in registers; writes the face flux and the bar state of field 0 at index fi.
template <class LAW, typename T, class S>
__device__ __forceinline__ void face_eval_r(S& s, int k, int L, const Vec<T, LAW::NC>& uR, const Vec<T, LAW::NC>& FR,
                                            const typename LAW::Aux& aR, T sR, int fi, const LawParamsT<T>& lp) {
  using V = Vec<T, LAW::NC>;
  constexpr int NC = LAW::NC;
  const V uL = s.u[L];
  const V FL = k ? s.fy[L] : s.fx[L];
  const typename LAW::Aux aL = s.aux[L];
  const T lam = LAW::lam(k, uL.v, aL, uR.v, aR, lp);
  V fb, fs, du;
  v_add<NC>(fs.v, FL.v, FR.v);
  v_sub<NC>(du.v, uR.v, uL.v);
  v_scale<NC>(fs.v, T(0.5), fs.v);
  v_fma<NC>(fb.v, T(-0.5) * lam, du.v, fs.v);
  Vec<T, LAW::kEntropy ? 2 : 1> bb;
  bb.v[0] = (lam > T(0)) ? T(0.5) * (uL.v[0] + uR.v[0]) - fdiv(FR.v[0] - FL.v[0], T(2) * lam)
                         : T(0.5) * (uL.v[0] + uR.v[0]);
  if constexpr (LAW::kEntropy) bb.v[1] = tmin(s.sig[L], sR);
  if (k == 0) { s.fbx[fi] = fb; s.bbx[fi] = bb; }
  else { s.fby[fi] = fb; s.bby[fi] = bb; }
}

// The whole stage for one tile of one problem instance.
// Unsparsified graph viscosity (Sec. 3.4 comparison mode): the low-order operator built on the
// dense DG-SEM differentiation matrix couples node j of a line of its element with every other
// node c of that line: c_jc = h w D[c][j] e_k, d_jc = lambda h w |D[c][j]| (|D[c][j]| = |D[j][c]| for
// c != j by summation by parts), bar state 1/2 (u_j + u_c) + sign(D[c][j]) (F_c - F_j) / (2 lambda).
// Accumulates, without the factor h w: vol = sum_c D[c][j] F_c, visc = sum_c lambda |D[c][j]| (u_c - u_j),
// lam = sum_c lambda |D[c][j]|, and the bar-state extremes of field 0 and the sigma minimum.
template <int P, class LAW, typename T, class S>
__device__ __forceinline__ void dense_line(const S& s, int k, int base, int stride, int j, const LawParamsT<T>& lp,
                                           T* vol, T* visc, T& lam, T& lo, T& hi, T& smin) {
  constexpr int n = P + 1, NC = LAW::NC;
  using V = Vec<T, NC>;
  const int me = base + j * stride;
  const V ui = s.u[me];
  const V Fi = (k == 0) ? s.fx[me] : s.fy[me];
  const typename LAW::Aux ai = s.aux[me];
#pragma unroll 1
  for (int c = 0; c < n; ++c) {
    const int sc = base + c * stride;
    const V Fc = (k == 0) ? s.fx[sc] : s.fy[sc];
    const T dcj = s.D[c * n + j];
#pragma unroll
    for (int q = 0; q < NC; ++q) vol[q] += dcj * Fc.v[q];
    if (c == j || dcj == T(0)) continue;  // pairs with c_jc = c_cj = 0 are not in the stencil
    const V uc = s.u[sc];
    const typename LAW::Aux ac = s.aux[sc];
    // the pair's Riemann problem runs along n_jc = -c_jc/|c_jc| = -sign(D[c][j]) e_k: node j is its
    // left state when D[c][j] < 0 (for the dense operator this need not match the nodes' order)
    const T l = (dcj < T(0)) ? LAW::lam(k, ui.v, ai, uc.v, ac, lp) : LAW::lam(k, uc.v, ac, ui.v, ai, lp);
    const T ad = fabs(dcj);
    lam += l * ad;
#pragma unroll
    for (int q = 0; q < NC; ++q) visc[q] += l * ad * (uc.v[q] - ui.v[q]);
    T bar = T(0.5) * (ui.v[0] + uc.v[0]);
    if (l > T(0)) bar += ((dcj > T(0)) ? T(1) : T(-1)) * fdiv(Fc.v[0] - Fi.v[0], T(2) * l);
    lo = tmin(lo, bar);
    hi = tmax(hi, bar);
    if constexpr (LAW::kEntropy) smin = tmin(smin, s.sig[sc]);
  }
}

// ELW selects elementwise limiting at compile time (its kernels are separate instantiations, so
// the subcell kernels carry none of its code).  SUBCELL: the configuration of the production runs
// (subcell limiting, smoothness indicator off) fixed at compile time, so that the kernel carries
// none of the other modes' branches.
template <int P, int TX, int TY, class LAW, typename T, bool ELW = false, bool DENSE = false, bool STATS = true,
          bool SUBCELL = false>
__device__ __forceinline__ void stage_body(TileSmem<P, TX, TY, LAW, T>& s, const Instance<T>& I, const Tables<T>& tab,
                                           const LawParamsT<T>& lp, int limiter_, const SmoothnessT<T>& si, int tile_x,
                                           int tile_y) {
  const int limiter = SUBCELL ? 2 : limiter_;
  const bool si_on = SUBCELL ? false : (si.on != 0);
  using G = TileGeom<P, TX, TY>;
  using V = Vec<T, LAW::NC>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const int t = threadIdx.x;

  // ---------------- A
  int le, a, b;
  long long g;
  NodeRec<LAW, T> own;
  const bool act = load_tile<P, TX, TY, LAW, false>(s, I, tab, lp, tile_x, tile_y, le, a, b, g, &own);
  __syncthreads();

  // ---------------- B: every face once.  Each node slot's thread evaluates the x face on its left
  // and the y face below it (its own side is still in registers); the NY + NX faces on the east
  // and north edges of the tile follow in one extra pass.
  if (t < G::NT) {
    const int row = (le / TX) * n + a, col = (le % TX) * n + b;
    // the node's own quantities are still in registers from phase A
    face_eval_r<LAW>(s, 0, Nbr<P, TX, TY>::left(t, b, row, col), own.u, own.fx, own.ax, own.sig, t, lp);
    face_eval_r<LAW>(s, 1, Nbr<P, TX, TY>::down(t, a, row, col), own.u, own.fy, own.ax, own.sig, t, lp);
  }
  for (int e2 = t; e2 < G::NY + G::NX; e2 += G::THREADS) {
    if (e2 < G::NY) {  // east edge: slot (row, NX-1) | halo E
      const int row = e2;
      const int L = G::slot(row, G::NX - 1), R = G::hE + row;
      face_eval_r<LAW>(s, 0, L, s.u[R], s.fx[R], s.aux[R], LAW::kEntropy ? s.sig[R] : T(0), G::NT + row, lp);
    } else {  // north edge: slot (NY-1, col) | halo N
      const int col = e2 - G::NY;
      const int L = G::slot(G::NY - 1, col), R = G::hN + col;
      face_eval_r<LAW>(s, 1, L, s.u[R], s.fy[R], s.aux[R], LAW::kEntropy ? s.sig[R] : T(0), G::NT + col, lp);
    }
  }
  __syncthreads();

  // ---------------- smoothness indicator (Sec. 4.4), when enabled: epsilon_K per element from the
  // Legendre coefficients of the limited field (separable nodal -> modal transform), s_K =
  // log10(||u - u-hat||^2 / ||u||^2) with u-hat dropping the modes of degree p in either variable
  const bool slot0 = (G::NT == G::THREADS) || (t < G::NT);
  if (si_on && limiter >= 2) {
    const int base = le * NN;
    if (slot0) {
      T c1 = T(0);
#pragma unroll
      for (int c = 0; c < n; ++c) c1 += s.Vinv[b * n + c] * s.u[base + a * n + c].v[0];
      s.alpha[t] = c1;
    }
    __syncthreads();
    T wgt = T(0);
    if (slot0) {
      T cc = T(0);
#pragma unroll
      for (int c = 0; c < n; ++c) cc += s.Vinv[a * n + c] * s.alpha[base + c * n + b];
      wgt = cc * cc * s.nrm[a] * s.nrm[b];
    }
    __syncthreads();
    if (slot0) s.alpha[t] = wgt;
    __syncthreads();
    if (slot0 && a == 0 && b == 0) {
      T tot = T(0), top = T(0);
      for (int i = 0; i < NN; ++i) {
        const T v = s.alpha[base + i];
        tot += v;
        if (i / n == P || i % n == P) top += v;
      }
      T e = T(0);
      if (tot > T(0) && top > T(0)) {
        const T sk = plog10(top / tot);
        e = (sk < si.s0 - si.kappa) ? T(0)
          : (sk > si.s0 + si.kappa) ? T(1)
          : T(0.5) + T(0.5) * psin(T(3.14159265358979323846) * (sk - si.s0) / (T(2) * si.kappa));
      }
      s.eps[le] = e;
    }
    __syncthreads();
  }

  // ---------------- C: residuals, low-order state, bounds
  // Every tile slot is computed (slots outside a ragged mesh edge hold valid ghost data); only
  // global-memory traffic is restricted to active nodes.  slot is false only for padding threads.
  const bool slot = (G::NT == G::THREADS) || (t < G::NT);
  const T dt = *I.dtT;
  const bool move = (dt > T(0)) && (dt < T(FLT_MAX));
  const T h = I.hT;
  const int row = (le / TX) * n + a, col = (le % TX) * n + b;
  const int me = le * NN + a * n + b;
  // the node's four faces: left and bottom at its own slot, right and top at the neighbour's (or
  // on the tile edge)
  const int ix = me, ixr = G::xface_right(me, b, row, col), iy = me, iyu = G::yface_up(me, a, row, col);
  const long long N = I.N;
  T uL[NC], rx[NC], ry[NC];
  T lo = T(0), hi = T(0), K = T(0), m = T(1), dtm = T(0);
  if (slot) {
    // the line contractions first: the node's own fluxes and its face fluxes are loaded after
    // them, so that fewer values are live at once
    T sx[NC], sy[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { sx[q] = T(0); sy[q] = T(0); }
    const int lx = le * NN + a * n, ly = le * NN + b;
#pragma unroll
    for (int c = 0; c < n; ++c) {
      const V Fxc = s.fx[lx + c];
      const V Fyc = s.fy[ly + c * n];
      const T dx = s.D[b * n + c], dy = s.D[a * n + c];
      v_fma<NC>(sx, dx, Fxc.v, sx);
      v_fma<NC>(sy, dy, Fyc.v, sy);
    }
    const V vu = s.u[me], vfx = s.fx[me], vfy = s.fy[me];
    const V fl = s.fbx[ix], fr = s.fbx[ixr], fd = s.fby[iy], fu = s.fby[iyu];
    const T wa = s.w[a], wb = s.w[b];
    const T hwa = h * wa, hwb = h * wb;
    m = h * h * wa * wb;
    dtm = move ? fdiv(dt, m) : T(0);
    T dvx[NC], dgx[NC], dvy[NC], dgy[NC];
    T dlo = vu.v[0], dhi = vu.v[0], dsig = T(0), dlam = T(0);
    if constexpr (DENSE) {
#pragma unroll
      for (int q = 0; q < NC; ++q) { dvx[q] = dgx[q] = dvy[q] = dgy[q] = T(0); }
      if constexpr (LAW::kEntropy) dsig = s.sig[me];
      dense_line<P, LAW>(s, 0, le * NN + a * n, 1, b, lp, dvx, dgx, dlam, dlo, dhi, dsig);
      dense_line<P, LAW>(s, 1, le * NN + b, n, a, lp, dvy, dgy, dlam, dlo, dhi, dsig);
    }
    T out[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {  // element-face terms of the high-order residual
      if (b == 0) sx[q] += vfx.v[q] - fl.v[q];
      if (b == P) sx[q] += fr.v[q] - vfx.v[q];
      if (a == 0) sy[q] += vfy.v[q] - fd.v[q];
      if (a == P) sy[q] += fu.v[q] - vfy.v[q];
    }
    T rHx[NC], rHy[NC], rLx[NC], rLy[NC], tq[NC];
    v_scale<NC>(rHx, -hwa, sx);
    v_scale<NC>(rHy, -hwb, sy);
    if constexpr (DENSE) {  // dense volume term and graph viscosity, element-face fluxes only
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        rLx[q] = hwa * (dvx[q] + dgx[q] + ((b == 0) ? fl.v[q] : T(0)) - ((b == P) ? fr.v[q] : T(0)));
        rLy[q] = hwb * (dvy[q] + dgy[q] + ((a == 0) ? fd.v[q] : T(0)) - ((a == P) ? fu.v[q] : T(0)));
      }
    } else {
      v_sub<NC>(tq, fr.v, fl.v);
      v_scale<NC>(rLx, -hwa, tq);
      v_sub<NC>(tq, fu.v, fd.v);
      v_scale<NC>(rLy, -hwb, tq);
    }
    v_add<NC>(tq, rLx, rLy);
    v_fma<NC>(uL, dtm, tq, vu.v);
    if (limiter == 0) {
      v_add<NC>(tq, rHx, rHy);
      v_fma<NC>(out, dtm, tq, vu.v);
    } else {
#pragma unroll
      for (int q = 0; q < NC; ++q) out[q] = uL[q];
    }
    v_sub<NC>(rx, rHx, rLx);
    v_sub<NC>(ry, rHy, rLy);
    if (limiter < 2 && act) {  // high-order target or low-order update only: done
#pragma unroll
      for (int q = 0; q < NC; ++q)
        I.uout[q * N + g] = (I.c0 == T(0)) ? out[q] : I.c0 * I.u0[q * N + g] + I.c1 * out[q];
    }
    const auto bl = s.bbx[ix], br = s.bbx[ixr], bd = s.bby[iy], bu = s.bby[iyu];
    if constexpr (DENSE) {  // in-element pairs from the dense lines, plus the element-face pairs
      lo = dlo;
      hi = dhi;
      if (b == 0) { lo = tmin(lo, bl.v[0]); hi = tmax(hi, bl.v[0]); }
      if (b == P) { lo = tmin(lo, br.v[0]); hi = tmax(hi, br.v[0]); }
      if (a == 0) { lo = tmin(lo, bd.v[0]); hi = tmax(hi, bd.v[0]); }
      if (a == P) { lo = tmin(lo, bu.v[0]); hi = tmax(hi, bu.v[0]); }
    } else {
      lo = tmin(tmin(vu.v[0], tmin(bl.v[0], br.v[0])), tmin(bd.v[0], bu.v[0]));
      hi = tmax(tmax(vu.v[0], tmax(bl.v[0], br.v[0])), tmax(bd.v[0], bu.v[0]));
    }
    if (si_on) {  // Eq. relaxed-bounds
      const T e = s.eps[le];
      lo = e * lo + (T(1) - e) * si.gmin;
      hi = e * hi + (T(1) - e) * si.gmax;
    }
    // K_i = min sigma over the node and its four neighbours = min over its four faces' minima
    if constexpr (LAW::kEntropy) {
      if constexpr (DENSE) {
        K = dsig;
        if (b == 0) K = tmin(K, bl.v[1]);
        if (b == P) K = tmin(K, br.v[1]);
        if (a == 0) K = tmin(K, bd.v[1]);
        if (a == P) K = tmin(K, bu.v[1]);
      } else {
        K = tmin(tmin(bl.v[1], br.v[1]), tmin(bd.v[1], bu.v[1]));
      }
    }
  }
  if (limiter < 2) return;  // uniform across the CTA
  if constexpr (ELW) {      // elementwise limiting (Sec. 4.1.2, 4.2.1)
    elementwise_update<P, TX, TY, LAW, T, DENSE>(s, I, lp, slot, act, move, g, le, me, a, b, uL, rx, ry, lo, hi, K, m, dt, dtm);
    return;
  }
  // ---------------- D: subcell fluxes and nodal alpha-tilde
  T xp[NC], xm[NC], yp[NC], ym[NC];
  T at = T(1);
  int iters = 0, caps = 0;
  if constexpr (32 % NN == 0) {
    // An element's nodes sit in NN consecutive lanes of one warp: the line prefix sums
    // r-bar = sum_{c <= b} r_c are warp scans (x lines: n consecutive lanes; y lines: stride n).
    // r-bar at face b-1/2 is taken from the neighbouring lane's inclusive sum, so both nodes of a
    // face use the same value.
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      T vx = rx[q], vy = ry[q];
#pragma unroll
      for (int d = 1; d < n; d <<= 1) {
        const T ox = __shfl_up_sync(0xffffffffu, vx, d, n);
        const T oy = __shfl_up_sync(0xffffffffu, vy, d * n, NN);
        if (b >= d) vx += ox;
        if (a >= d) vy += oy;
      }
      const T px = __shfl_up_sync(0xffffffffu, vx, 1, n);
      const T py = __shfl_up_sync(0xffffffffu, vy, n, NN);
      xm[q] = (b > 0) ? px : T(0);
      ym[q] = (a > 0) ? py : T(0);
      xp[q] = (b == P) ? T(0) : vx;
      yp[q] = (a == P) ? T(0) : vy;
    }
  } else {
    __syncthreads();  // all reads of F_x, F_y done
    if (slot) {
      V vrx, vry;
#pragma unroll
      for (int q = 0; q < NC; ++q) { vrx.v[q] = rx[q]; vry.v[q] = ry[q]; }
      s.fx[me] = vrx;
      s.fy[me] = vry;
    }
    __syncthreads();
    if (slot) {
#pragma unroll
      for (int q = 0; q < NC; ++q) { xm[q] = T(0); ym[q] = T(0); }
      const int lx = le * NN + a * n, ly = le * NN + b;
#pragma unroll
      for (int c = 0; c < P; ++c) {
        if (c < b) {
          const V r = s.fx[lx + c];
#pragma unroll
          for (int q = 0; q < NC; ++q) xm[q] += r.v[q];
        }
        if (c < a) {
          const V r = s.fy[ly + c * n];
#pragma unroll
          for (int q = 0; q < NC; ++q) ym[q] += r.v[q];
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        xp[q] = (b == P) ? T(0) : xm[q] + rx[q];
        yp[q] = (a == P) ? T(0) : ym[q] + ry[q];
      }
    }
  }
  if (slot) {
    if (move) {
      const T c1 = xp[0], c2 = -xm[0], c3 = yp[0], c4 = -ym[0];
      const T Pp = tmax(c1, T(0)) + tmax(c2, T(0)) + tmax(c3, T(0)) + tmax(c4, T(0));
      const T Pm = tmin(c1, T(0)) + tmin(c2, T(0)) + tmin(c3, T(0)) + tmin(c4, T(0));
      const T mdt = fdiv(m, dt);
      const T Qp = tmax(T(0), mdt * (hi - uL[0]));
      const T Qm = tmin(T(0), mdt * (lo - uL[0]));
      const T Rp = (Pp > T(0)) ? tmin(T(1), fdiv(Qp, Pp)) : T(1);
      const T Rm = (Pm < T(0)) ? tmin(T(1), fdiv(Qm, Pm)) : T(1);
      at = tmin(Rp, Rm);
      if constexpr (LAW::kEntropy)
        at = entropy_limit<LAW>(uL, K * (T(1) + Prec<T>::entropy_margin), xp, xm, yp, ym, T(4) * dtm, at, lp, iters, caps);
    }
    s.alpha[me] = at;
    if (I.dbg_lo && act) {
      I.dbg_lo[g] = (double)lo;
      I.dbg_hi[g] = (double)hi;
      I.dbg_K[g] = (double)K;
      I.dbg_alpha[g] = (double)at;
    }
  }
  T u0[NC];  // u^n for the RK combination; its latency overlaps the barrier
  if (act && I.c0 != T(0)) {
#pragma unroll
    for (int q = 0; q < NC; ++q) u0[q] = I.u0[q * N + g];
  }
  __syncthreads();
  // ---------------- E: face coefficients and limited update
  T fe[NC];
  int nudged = 0;
  if (slot) {
    const T axp = (b < P) ? tmin(at, s.alpha[me + 1]) : T(0);
    const T axm = (b > 0) ? tmin(at, s.alpha[me - 1]) : T(0);
    const T ayp = (a < P) ? tmin(at, s.alpha[me + n]) : T(0);
    const T aym = (a > 0) ? tmin(at, s.alpha[me - n]) : T(0);
    T acc[NC];
    v_scale<NC>(acc, axp, xp);
    v_fma<NC>(acc, -axm, xm, acc);
    v_fma<NC>(acc, ayp, yp, acc);
    v_fma<NC>(acc, -aym, ym, acc);
    v_fma<NC>(fe, dtm, acc, uL);
    if constexpr (sizeof(T) == 4) {
      if (!(fe[0] >= lo && fe[0] <= hi)) {  // rare: the rounding scale only where it is needed
        const T mag = stencil_scale<P, TX, TY, DENSE>(s, me, le, a, b, row, col) + fabs(uL[0]) +
                      tmax(fabs(lo), fabs(hi)) +
                      dtm * (fabs(axp * xp[0]) + fabs(axm * xm[0]) + fabs(ayp * yp[0]) + fabs(aym * ym[0]));
        nudged = accept_rounded(fe[0], lo, hi, mag);
      }
    }
    if (act) {
      T res[NC];
      if (I.c0 == T(0)) {
#pragma unroll
        for (int q = 0; q < NC; ++q) res[q] = fe[q];
      } else {  // the SSP-RK3 combination c0 u^n + c1 u^FE
        v_scale<NC>(res, I.c1, fe);
        v_fma<NC>(res, I.c0, u0, res);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) I.uout[q * N + g] = res[q];
    }
  }
  if (STATS && I.stats) {  // statistics: compiled only into the statistics kernels
    Vec<T, NC> vf;
#pragma unroll
    for (int q = 0; q < NC; ++q) vf.v[q] = fe[q];
    stage_stats<P, TX, TY, LAW, T, DENSE>(s, I, lp, act && move, vf, lo, hi, K, caps, iters, act ? nudged : 0, me, a,
                                          b, row, col);
  }
}

// STATS: a kernel with the per-stage statistics (launched when they are on); the timed kernels
// carry none of their code.
template <int P, int TX, int TY, class LAW, typename T, bool ELW = false, bool DENSE = false, bool STATS = false,
          bool SUBCELL = false>
__global__ void __launch_bounds__(TileGeom<P, TX, TY>::THREADS, TileGeom<P, TX, TY>::MINB)
k_stage(const StageLaunch<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<TileSmem<P, TX, TY, LAW, T>*>(smem_raw);
  const int tiles_x = (A.inst.nx + TX - 1) / TX;
  const int tile_y = blockIdx.x / tiles_x, tile_x = blockIdx.x - tile_y * tiles_x;
  stage_body<P, TX, TY, LAW, T, ELW, DENSE, STATS || ELW || DENSE, SUBCELL>(s, A.inst, A.tab, A.lp, A.limiter, A.si,
                                                                              tile_x, tile_y);
}

// Copy the instance descriptor of this CTA's task into shared memory (all threads help).
template <typename T>
__device__ __forceinline__ void load_instance(Instance<T>& dst, const Instance<T>* src) {
  static_assert(sizeof(Instance<T>) % 4 == 0, "instance size");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Instance<T>) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// Batched stage: CTA blockIdx.x runs task (instance, tile) of the task table; all tasks of one
// launch share P, the tile shape, law and precision.
template <int P, int TX, int TY, class LAW, typename T, bool ELW = false, bool STATS = false, bool SUBCELL = false>
__global__ void __launch_bounds__(TileGeom<P, TX, TY>::THREADS, TileGeom<P, TX, TY>::MINB)
k_stage_batch(const BatchLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<TileSmem<P, TX, TY, LAW, T>*>(smem_raw);
  __shared__ Instance<T> sI;
  const int2 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  const int tiles_x = (sI.nx + TX - 1) / TX;
  const int tile_y = task.y / tiles_x, tile_x = task.y - tile_y * tiles_x;
  stage_body<P, TX, TY, LAW, T, ELW, false, STATS || ELW, SUBCELL>(s, sI, B.tab, B.lp, B.limiter, B.si, tile_x, tile_y);
}

// CFL bound of Eq. cfl-low per node, m_i / (2 sum_{j != i} d-hat_ij) with d-hat = (h w / 2) lambda on
// the node's four faces, min-reduced into *out_bits (positive doubles order like their bit patterns).
// Same tile machinery as the stage kernel: node quantities once per node, lambda once per face.
template <int P, int TX, int TY, class LAW, typename T, bool DENSE = false>
__device__ __forceinline__ void dt_body(DtSmem<P, TX, TY, LAW, T>& s, const Instance<T>& I, const Tables<T>& tab,
                                        const LawParamsT<T>& lp, int tile_x, int tile_y, unsigned long long* out_bits) {
  using G = TileGeom<P, TX, TY>;
  using V = Vec<T, LAW::NC>;
  constexpr int n = P + 1;
  const int t = threadIdx.x;
  int le, a, b;
  long long g;
  const bool act = load_tile<P, TX, TY, LAW, true>(s, I, tab, lp, tile_x, tile_y, le, a, b, g);
  __syncthreads();
  T* lamx = s.lamx;
  T* lamy = s.lamy;
  if (t < G::NT) {
    const int row = (le / TX) * n + a, col = (le % TX) * n + b;
    const V uR = s.u[t];
    const typename LAW::Aux aR = s.aux[t];
    const int L = Nbr<P, TX, TY>::left(t, b, row, col), D = Nbr<P, TX, TY>::down(t, a, row, col);
    const V uL = s.u[L], uD = s.u[D];
    lamx[t] = LAW::lam(0, uL.v, s.aux[L], uR.v, aR, lp);
    lamy[t] = LAW::lam(1, uD.v, s.aux[D], uR.v, aR, lp);
  }
  for (int e2 = t; e2 < G::NY + G::NX; e2 += G::THREADS) {
    if (e2 < G::NY) {
      const int L = G::slot(e2, G::NX - 1), R = G::hE + e2;
      const V uL = s.u[L], uR = s.u[R];
      lamx[G::NT + e2] = LAW::lam(0, uL.v, s.aux[L], uR.v, s.aux[R], lp);
    } else {
      const int col = e2 - G::NY;
      const int L = G::slot(G::NY - 1, col), R = G::hN + col;
      const V uL = s.u[L], uR = s.u[R];
      lamy[G::NT + col] = LAW::lam(1, uL.v, s.aux[L], uR.v, s.aux[R], lp);
    }
  }
  __syncthreads();
  // per-node bound in the stage precision; the min is exact in any precision, and one
  // conversion per block hands it to the float64 accumulator
  const T big = T(FLT_MAX);
  T val = big;
  if (act) {
    const int row = (le / TX) * n + a, col = (le % TX) * n + b;
    const int me = le * (n * n) + a * n + b;
    const int ix = me, ixr = G::xface_right(me, b, row, col), iy = me, iyu = G::yface_up(me, a, row, col);
    const T h = I.hT;
    const T wa = s.w[a], wb = s.w[b];
    T sumd = T(0.5) * h * wa * (lamx[ix] + lamx[ixr]) + T(0.5) * h * wb * (lamy[iy] + lamy[iyu]);
    if constexpr (DENSE) {  // element-face pairs as above; every in-element pair of the dense lines
      constexpr int NN = n * n;
      sumd = T(0.5) * h * wa * (((b == 0) ? lamx[ix] : T(0)) + ((b == P) ? lamx[ixr] : T(0))) +
             T(0.5) * h * wb * (((a == 0) ? lamy[iy] : T(0)) + ((a == P) ? lamy[iyu] : T(0)));
      const int me = le * NN + a * n + b;
      const V ui = s.u[me];
      const typename LAW::Aux ai = s.aux[me];
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        if (c != b && s.D[c * n + b] != T(0)) {
          const int sc = le * NN + a * n + c;
          const V uc = s.u[sc];
          const T l = (s.D[c * n + b] < T(0)) ? LAW::lam(0, ui.v, ai, uc.v, s.aux[sc], lp)
                                               : LAW::lam(0, uc.v, s.aux[sc], ui.v, ai, lp);
          sumd += h * wa * l * fabs(s.D[c * n + b]);
        }
        if (c != a && s.D[c * n + a] != T(0)) {
          const int sc = le * NN + c * n + b;
          const V uc = s.u[sc];
          const T l = (s.D[c * n + a] < T(0)) ? LAW::lam(1, ui.v, ai, uc.v, s.aux[sc], lp)
                                               : LAW::lam(1, uc.v, s.aux[sc], ui.v, ai, lp);
          sumd += h * wb * l * fabs(s.D[c * n + a]);
        }
      }
    }
    if (sumd > T(0)) val = fdiv(h * h * wa * wb, T(2) * sumd);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val = tmin(val, __shfl_xor_sync(0xffffffffu, val, o));
  __shared__ T red[32];
  if ((t & 31) == 0) red[t >> 5] = val;
  __syncthreads();
  if (t < 32) {
    val = (t < G::THREADS / 32) ? red[t] : big;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val = tmin(val, __shfl_xor_sync(0xffffffffu, val, o));
    if (t == 0 && val < big) atomicMin(out_bits, (unsigned long long)__double_as_longlong((double)val));
  }
}

template <int P, int TX, int TY, class LAW, typename T, bool DENSE = false>
__global__ void __launch_bounds__(TileGeom<P, TX, TY>::THREADS, TileGeom<P, TX, TY>::MINB)
k_dt(const StageLaunch<T> A, unsigned long long* out_bits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<DtSmem<P, TX, TY, LAW, T>*>(smem_raw);
  const int tiles_x = (A.inst.nx + TX - 1) / TX;
  const int tile_y = blockIdx.x / tiles_x, tile_x = blockIdx.x - tile_y * tiles_x;
  dt_body<P, TX, TY, LAW, T, DENSE>(s, A.inst, A.tab, A.lp, tile_x, tile_y, out_bits);
}

template <int P, int TX, int TY, class LAW, typename T>
__global__ void __launch_bounds__(TileGeom<P, TX, TY>::THREADS, TileGeom<P, TX, TY>::MINB)
k_dt_batch(const BatchLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<DtSmem<P, TX, TY, LAW, T>*>(smem_raw);
  __shared__ Instance<T> sI;
  const int2 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  const int tiles_x = (sI.nx + TX - 1) / TX;
  const int tile_y = task.y / tiles_x, tile_x = task.y - tile_y * tiles_x;
  dt_body<P, TX, TY, LAW, T>(s, sI, B.tab, B.lp, tile_x, tile_y, B.bits + task.x);
}

// ---------------------------------------------------------------- single-launch batches
// One launch over the tiles of every instance of a batch, whatever their degree: each CTA switches
// on its task's degree into the stage (or time-step) body of that degree with its default tile
// shape.  Every default shape has at most 256 nodes, so one block size and one register budget
// (64 registers, 4 CTAs per SM) serve all degrees; the dynamic shared memory is the largest
// degree's.  Tasks are ordered by decreasing degree (the costliest tiles first).
template <int P>
struct DefaultTile {
  static constexpr int TX = kTiles[P][0].tx, TY = kTiles[P][0].ty;
  static_assert(TileGeom<P, TX, TY>::THREADS == 256, "single-launch batches need 256-thread default tiles");
};

template <int P, class LAW, typename T, bool DT>
__device__ __forceinline__ void batch_all_body(unsigned char* smem_raw, const Instance<T>& I, const BatchAllLaunch<T>& B,
                                               int tile, int inst) {
  constexpr int TX = DefaultTile<P>::TX, TY = DefaultTile<P>::TY;
  const int tiles_x = (I.nx + TX - 1) / TX;
  const int tile_y = tile / tiles_x, tile_x = tile - tile_y * tiles_x;
  if constexpr (DT) {
    dt_body<P, TX, TY, LAW, T>(*reinterpret_cast<DtSmem<P, TX, TY, LAW, T>*>(smem_raw), I, B.tabs[P], B.lp, tile_x, tile_y,
                               B.bits + inst);
  } else {
    stage_body<P, TX, TY, LAW, T, false, false, false, true>(*reinterpret_cast<TileSmem<P, TX, TY, LAW, T>*>(smem_raw), I,
                                                             B.tabs[P], B.lp, 2, B.si, tile_x, tile_y);
  }
}

template <class LAW, typename T, bool DT>
__global__ void __launch_bounds__(256, 4) k_batch_all(const BatchAllLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Instance<T> sI;
  const int4 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  switch (task.z) {
    case 1: batch_all_body<1, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    case 2: batch_all_body<2, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    case 3: batch_all_body<3, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    case 4: batch_all_body<4, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    case 5: batch_all_body<5, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    case 6: batch_all_body<6, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
    default: batch_all_body<7, LAW, T, DT>(smem_raw, sI, B, task.y, task.x); break;
  }
}

template <class LAW, typename T, bool DT>
constexpr size_t batch_all_smem() {
  size_t m = 0;
#define SIDP_SMEM_P(P)                                                                                       \
  {                                                                                                          \
    const size_t v = DT ? sizeof(DtSmem<P, DefaultTile<P>::TX, DefaultTile<P>::TY, LAW, T>)                  \
                        : sizeof(TileSmem<P, DefaultTile<P>::TX, DefaultTile<P>::TY, LAW, T>);               \
    m = v > m ? v : m;                                                                                       \
  }
  SIDP_SMEM_P(1) SIDP_SMEM_P(2) SIDP_SMEM_P(3) SIDP_SMEM_P(4) SIDP_SMEM_P(5) SIDP_SMEM_P(6) SIDP_SMEM_P(7)
#undef SIDP_SMEM_P
  return m;
}

template <class LAW, typename T>
cudaError_t launch_batch_all_law(const BatchAllLaunch<T>& B, bool dt, cudaStream_t s) {
  constexpr size_t smem = batch_all_smem<LAW, T, false>(), smem_dt = batch_all_smem<LAW, T, true>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_batch_all<LAW, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_batch_all<LAW, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dt);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (B.ntasks <= 0) return cudaSuccess;
  if (dt) k_batch_all<LAW, T, true><<<(unsigned)B.ntasks, 256, smem_dt, s>>>(B);
  else k_batch_all<LAW, T, false><<<(unsigned)B.ntasks, 256, smem, s>>>(B);
  return cudaGetLastError();
}

template <int P, int TX, int TY, class LAW, typename T, bool ELW = false, bool DENSE = false, bool STATS = false,
          bool SUBCELL = false>
cudaError_t launch_tile(const StageLaunch<T>& a, unsigned long long* dt_bits, cudaStream_t s) {
  using G = TileGeom<P, TX, TY>;
  constexpr size_t smem = sizeof(TileSmem<P, TX, TY, LAW, T>);
  constexpr size_t smem_dt = sizeof(DtSmem<P, TX, TY, LAW, T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_stage<P, TX, TY, LAW, T, ELW, DENSE, STATS, SUBCELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_dt<P, TX, TY, LAW, T, DENSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dt);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  const long long tiles = (long long)((a.inst.nx + TX - 1) / TX) * ((a.inst.ny + TY - 1) / TY);
  if (tiles <= 0) return cudaSuccess;
  if (dt_bits) k_dt<P, TX, TY, LAW, T, DENSE><<<(unsigned)tiles, G::THREADS, smem_dt, s>>>(a, dt_bits);
  else k_stage<P, TX, TY, LAW, T, ELW, DENSE, STATS, SUBCELL><<<(unsigned)tiles, G::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int TX, int TY, class LAW, typename T, bool ELW = false, bool STATS = false, bool SUBCELL = false>
cudaError_t launch_batch_tile(const BatchLaunch<T>& B, bool dt, cudaStream_t s) {
  using G = TileGeom<P, TX, TY>;
  constexpr size_t smem = sizeof(TileSmem<P, TX, TY, LAW, T>);
  constexpr size_t smem_dt = sizeof(DtSmem<P, TX, TY, LAW, T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_stage_batch<P, TX, TY, LAW, T, ELW, STATS, SUBCELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_dt_batch<P, TX, TY, LAW, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dt);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (B.ntasks <= 0) return cudaSuccess;
  if (dt) k_dt_batch<P, TX, TY, LAW, T><<<(unsigned)B.ntasks, G::THREADS, smem_dt, s>>>(B);
  else k_stage_batch<P, TX, TY, LAW, T, ELW, STATS, SUBCELL><<<(unsigned)B.ntasks, G::THREADS, smem, s>>>(B);
  return cudaGetLastError();
}

}  // namespace sidp
