// Line-parallel stage kernel: the forward-Euler update of Sec. 4 (Eq. subcell-fct / convex-fct)
// with subcell limiting and the SSP-RK3 combination of Sec. 5, one thread per element line.
//
// A CTA owns a tile of EX x EY elements.  Thread j of element K is at once the thread of row j
// (nodes (j, b), b = 0..p) and of column j (nodes (a, j), a = 0..p) of K.  Every index inside an
// element is then a compile-time constant of the thread's unrolled loops: the line contractions
// with D_1D, the subcell faces along the line, the element-face terms and the prefix sums of the
// subcell fluxes run in registers, with D_1D and the weights as constant operands.
//   A  each thread loads its row (vector loads: a row of an element is contiguous per field),
//      computes the per-node quantities, and stores state, per-node quantities and sigma in
//      shared memory; halo slots (the traces across the tile's edges) as in the node kernel.
//   B  column role: the column's nodes and its two neighbours across the element's faces are
//      read from shared memory; the y faces (Lax-Friedrichs flux on element faces, Eq.
//      lax-friedrichs; sparsified low-order operator on subcell faces, Eq. didp / Eq. dij), the
//      y contraction, r^H_y and r^L_y, the bar-state bounds and the prefix sums along the
//      column go to shared memory for the row threads.
//   C  row role: the same along x (the row re-read from shared memory by vector loads).
//   D  per node of the row: u^L, the local bounds (Sec. 4.1.1, 4.3), Zalesak's coefficient and
//      the entropy line search (Sec. 4.1.3, 4.2) -> alpha-tilde, stored per node.
//   E  face coefficients alpha = min of the two nodes' alpha-tilde, the limited update, the
//      post-round acceptance of the float32 store, the RK combination, vector stores.
// Element faces are evaluated by both adjacent lines (each from the same left and right states
// in the same order, hence bit-identical), so the update stays conservative up to the rounding
// of the final sums; no face values are exchanged between threads.
#pragma once
#include "sidp_kernels.cuh"

namespace sidp {

template <int P, int EX, int EY>
struct LineGeom {
  static constexpr int n = P + 1, NN = n * n, NE = EX * EY;
  static constexpr int NL = NE * n;  // element lines: the working threads
  static constexpr int THREADS = ((NL + 31) / 32) * 32;
  static constexpr int NX = EX * n, NY = EY * n;
  // Shared-memory layout of an element's nodes.  p = 3: the rows of element le are rotated by
  // (le / 2) mod 4, so that both a warp's row accesses (16-byte vectors of 8 consecutive
  // elements' rows) and its column accesses (one value per lane of the same row of 8 elements)
  // fall in distinct banks.  Other degrees: rows in order, the element stride padded against the
  // column accesses' conflicts.
  static constexpr bool SWZ = (n == 4);
  static constexpr int SE = SWZ ? NN : NN + (NN == 4 ? 2 : NN == 64 ? 8 : 0);
  // slot of node (a, 0) of element le
  __device__ __forceinline__ static int rs(int le, int a) {
    if constexpr (SWZ) return le * SE + n * ((a + (le >> 1)) & 3);
    else return le * SE + n * a;
  }
  // a warp holds whole tile rows of elements: the west and east neighbours of a row come from the
  // adjacent lanes' registers
  static constexpr bool XSHFL = (EX * n == 32);
  static constexpr int NTP = ((NE * SE + 3) / 4) * 4;
  static constexpr int NH = 2 * NX + 2 * NY;  // halo slots: W[NY], E[NY], S[NX], N[NX]
  static constexpr int hW = NTP, hE = NTP + NY, hS = NTP + 2 * NY, hN = NTP + 2 * NY + NX;
  static constexpr int NS = ((NTP + NH + 3) / 4) * 4;
};

template <class LAW, typename T>
struct AuxWords {
  static constexpr int value = sizeof(typename LAW::Aux) >= sizeof(T) ? int(sizeof(typename LAW::Aux) / sizeof(T)) : 0;
};

template <int P, int EX, int EY, class LAW, typename T>
struct LineSmem {
  using G = LineGeom<P, EX, EY>;
  static constexpr int NC = LAW::NC, NA = AuxWords<LAW, T>::value;
  // stage input, per-node quantities and sigma of every node and halo slot (phases A-E)
  T u[NC][G::NS];
  T aux[NA > 0 ? NA : 1][G::NS];
  T sig[LAW::kEntropy ? G::NS : 4];
  // column -> row: r^L_y, the y prefix sum at the face above the node, y-face bounds
  T rly[NC][G::NTP];
  T sy[NC][G::NTP];
  T lo[G::NTP];
  T hi[G::NTP];
  T K[LAW::kEntropy ? G::NTP : 4];
  T alpha[G::NTP];
};

// Widest vector (elements of T, at most 16 bytes) that divides a line of n values; lines start
// at multiples of n elements in global memory and at multiples of 4 (n = 4, 8) or n in shared
// memory, so the vector accesses are aligned.
template <int n, typename T>
struct LineVec {
  static constexpr int W16 = 16 / int(sizeof(T));
  static constexpr int W = (n % W16 == 0) ? W16 : (n % 2 == 0 && sizeof(T) == 4) ? 2 : 1;
};

template <int n, typename T>
__device__ __forceinline__ void ld_line(const T* p, T* v) {
  constexpr int W = LineVec<n, T>::W;
  if constexpr (W == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 4) {
      const float4 r = *reinterpret_cast<const float4*>(p + i);
      v[i] = r.x; v[i + 1] = r.y; v[i + 2] = r.z; v[i + 3] = r.w;
    }
  } else if constexpr (W == 2 && sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < n; i += 2) {
      const double2 r = *reinterpret_cast<const double2*>(p + i);
      v[i] = r.x; v[i + 1] = r.y;
    }
  } else if constexpr (W == 2) {
#pragma unroll
    for (int i = 0; i < n; i += 2) {
      const float2 r = *reinterpret_cast<const float2*>(p + i);
      v[i] = r.x; v[i + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) v[i] = p[i];
  }
}

template <int n, typename T>
__device__ __forceinline__ void st_line(T* p, const T* v) {
  constexpr int W = LineVec<n, T>::W;
  if constexpr (W == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else if constexpr (W == 2 && sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < n; i += 2) *reinterpret_cast<double2*>(p + i) = make_double2(v[i], v[i + 1]);
  } else if constexpr (W == 2) {
#pragma unroll
    for (int i = 0; i < n; i += 2) *reinterpret_cast<float2*>(p + i) = make_float2(v[i], v[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) p[i] = v[i];
  }
}

// Table entry at a runtime index i < n (unrolled selection: no indexed parameter access).
template <int n, typename T>
__device__ __forceinline__ T pick(const T* tab, int i) {
  T v = tab[0];
#pragma unroll
  for (int c = 1; c < n; ++c)
    if (i == c) v = tab[c];
  return v;
}

// The quantities of one node kept by a line: state, per-node quantities, sigma.
template <class LAW, typename T>
struct LNode {
  T u[LAW::NC];
  typename LAW::Aux ax;
  T s;
};

template <class LAW, typename T, class S>
__device__ __forceinline__ void ld_node(const S& s, int slot, LNode<LAW, T>& nd) {
  constexpr int NA = AuxWords<LAW, T>::value;
#pragma unroll
  for (int q = 0; q < LAW::NC; ++q) nd.u[q] = s.u[q][slot];
  if constexpr (NA > 0) {
    T* aw = reinterpret_cast<T*>(&nd.ax);
#pragma unroll
    for (int k = 0; k < NA; ++k) aw[k] = s.aux[k][slot];
  }
  nd.s = LAW::kEntropy ? s.sig[slot] : T(0);
}

template <class LAW, typename T, class S, bool SIG = true>
__device__ __forceinline__ void st_node(S& s, int slot, const T* uu, const typename LAW::Aux& ax, T sg) {
  constexpr int NA = AuxWords<LAW, T>::value;
#pragma unroll
  for (int q = 0; q < LAW::NC; ++q) s.u[q][slot] = uu[q];
  if constexpr (NA > 0) {
    const T* aw = reinterpret_cast<const T*>(&ax);
#pragma unroll
    for (int k = 0; k < NA; ++k) s.aux[k][slot] = aw[k];
  }
  if constexpr (LAW::kEntropy && SIG) s.sig[slot] = sg;
}

// dst = src of lane (lane + delta) (all 32 lanes call it; lanes whose source is outside the warp
// get an unspecified node and overwrite it)
template <class LAW, typename T>
__device__ __forceinline__ void shfl_node(const LNode<LAW, T>& src, LNode<LAW, T>& dst, int delta) {
  constexpr int NA = AuxWords<LAW, T>::value;
  auto sh = [&](T v) {
    return delta > 0 ? __shfl_down_sync(0xffffffffu, v, (unsigned)delta) : __shfl_up_sync(0xffffffffu, v, (unsigned)(-delta));
  };
#pragma unroll
  for (int q = 0; q < LAW::NC; ++q) dst.u[q] = sh(src.u[q]);
  if constexpr (NA > 0) {
    const T* as = reinterpret_cast<const T*>(&src.ax);
    T* ad = reinterpret_cast<T*>(&dst.ax);
#pragma unroll
    for (int k = 0; k < NA; ++k) ad[k] = sh(as[k]);
  }
  dst.s = LAW::kEntropy ? sh(src.s) : T(0);
}

template <class LAW, typename T>
__device__ __forceinline__ void node_aux(const T* uu, T x, T y, typename LAW::Aux& ax, const LawParamsT<T>& lp) {
  if constexpr (HasPosition<LAW>::value) LAW::aux_at(uu, x, y, ax, lp);
  else LAW::aux(uu, ax, lp);
}

// Face along +e_K between the states L and R: the face flux 1/2 (F_L + F_R) - lambda/2 (u_R - u_L),
// the bar state of the limited field and min(sigma_L, sigma_R).  The same arithmetic, in the same
// order, as the node kernel's face evaluation.
template <int K, class LAW, typename T>
__device__ __forceinline__ void face_lr(const LNode<LAW, T>& L, const T* FL, const LNode<LAW, T>& R, const T* FR,
                                        const LawParamsT<T>& lp, T* fb, T& bar, T& smin) {
  constexpr int NC = LAW::NC;
  const T lam = LAW::lam(K, L.u, L.ax, R.u, R.ax, lp);
  T fs[NC], du[NC];
  v_add<NC>(fs, FL, FR);
  v_sub<NC>(du, R.u, L.u);
  v_scale<NC>(fs, T(0.5), fs);
  v_fma<NC>(fb, T(-0.5) * lam, du, fs);
  bar = (lam > T(0)) ? T(0.5) * (L.u[0] + R.u[0]) - fdiv(FR[0] - FL[0], T(2) * lam) : T(0.5) * (L.u[0] + R.u[0]);
  smin = LAW::kEntropy ? tmin(L.s, R.s) : T(0);
}

// One direction of one element line: the n nodes and the two neighbours across the element's faces
// (already loaded), the faces along the line, the contraction and the residuals.  Outputs per node:
// r^L (rl), the bounds from the node and its two faces on this line (lo, hi, K), and the inclusive
// prefix sums of r^H - r^L at the P interior faces (S).
template <int P, int DIR, class LAW, typename T>
__device__ __forceinline__ void line_residuals(const Tables<T>& tab, const LawParamsT<T>& lp, const LNode<LAW, T>* nd,
                                               const LNode<LAW, T>& lft, const LNode<LAW, T>& rgt, T hw,
                                               T (*rl)[LAW::NC], T* lo, T* hi, T* K, T (*S)[LAW::NC]) {
  constexpr int n = P + 1, NC = LAW::NC;
  T F[n][NC];
#pragma unroll
  for (int c = 0; c < n; ++c) LAW::flux(nd[c].u, nd[c].ax, DIR, F[c], lp);
  // contraction with D_1D along the line
  T sx[n][NC];
#pragma unroll
  for (int b = 0; b < n; ++b) {
#pragma unroll
    for (int q = 0; q < NC; ++q) sx[b][q] = T(0);
#pragma unroll
    for (int c = 0; c < n; ++c) v_fma<NC>(sx[b], tab.D[b * n + c], F[c], sx[b]);
  }
  // faces: f[0] left element face, f[1..P] subcell faces, f[n] right element face
  T fb[n + 1][NC], bar[n + 1], sm[n + 1];
  {
    T Fl[NC], Fr[NC];
    LAW::flux(lft.u, lft.ax, DIR, Fl, lp);
    LAW::flux(rgt.u, rgt.ax, DIR, Fr, lp);
    face_lr<DIR, LAW>(lft, Fl, nd[0], F[0], lp, fb[0], bar[0], sm[0]);
    face_lr<DIR, LAW>(nd[P], F[P], rgt, Fr, lp, fb[n], bar[n], sm[n]);
  }
#pragma unroll
  for (int c = 1; c < n; ++c) face_lr<DIR, LAW>(nd[c - 1], F[c - 1], nd[c], F[c], lp, fb[c], bar[c], sm[c]);
  // element-face terms of the high-order residual (strong form, Eq. ho-update)
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    sx[0][q] += F[0][q] - fb[0][q];
    sx[P][q] += fb[n][q] - F[P][q];
  }
  T acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = T(0);
#pragma unroll
  for (int b = 0; b < n; ++b) {
    T rH[NC], tq[NC], r[NC];
    v_scale<NC>(rH, -hw, sx[b]);
    v_sub<NC>(tq, fb[b + 1], fb[b]);
    v_scale<NC>(rl[b], -hw, tq);
    v_sub<NC>(r, rH, rl[b]);
    lo[b] = tmin(nd[b].u[0], tmin(bar[b], bar[b + 1]));
    hi[b] = tmax(nd[b].u[0], tmax(bar[b], bar[b + 1]));
    K[b] = tmin(sm[b], sm[b + 1]);
    if (b < P) {
      v_add<NC>(acc, acc, r);
#pragma unroll
      for (int q = 0; q < NC; ++q) S[b][q] = acc[q];
    }
  }
}

// Shared-memory slots of the neighbours of line j of element le (tile position tx, ty) across the
// element's faces: the west/east neighbours of row node (j, 0) / (j, P) and the south/north
// neighbours of column node (0, j) / (P, j) -- in the tile or in its halo.
template <int P, int EX, int EY>
struct LineNbr {
  using G = LineGeom<P, EX, EY>;
  static constexpr int n = P + 1;
  __device__ __forceinline__ static int west(int le, int tx, int ty, int j) {
    return (tx > 0) ? G::rs(le - 1, j) + P : G::hW + ty * n + j;
  }
  __device__ __forceinline__ static int east(int le, int tx, int ty, int j) {
    return (tx < EX - 1) ? G::rs(le + 1, j) : G::hE + ty * n + j;
  }
  __device__ __forceinline__ static int south(int le, int tx, int ty, int j) {
    return (ty > 0) ? G::rs(le - EX, P) + j : G::hS + tx * n + j;
  }
  __device__ __forceinline__ static int north(int le, int tx, int ty, int j) {
    return (ty < EY - 1) ? G::rs(le + EX, 0) + j : G::hN + tx * n + j;
  }
};

// Limited field's stencil scale |u_i| + 2 max |u_j| of row node (j, b) from the stage input in
// shared memory (the rare post-round acceptance path only).
template <int P, int EX, int EY, class S>
__device__ __forceinline__ auto line_stencil_scale(const S& s, int le, int tx, int ty, int j, int b) {
  using G = LineGeom<P, EX, EY>;
  using N4 = LineNbr<P, EX, EY>;
  constexpr int n = P + 1;
  const int me = G::rs(le, j) + b;
  const int l = (b > 0) ? me - 1 : N4::west(le, tx, ty, j);
  const int r = (b < P) ? me + 1 : N4::east(le, tx, ty, j);
  const int d = (j > 0) ? G::rs(le, j - 1) + b : N4::south(le, tx, ty, b);
  const int u = (j < P) ? G::rs(le, j + 1) + b : N4::north(le, tx, ty, b);
  auto S0 = tmax(tmax(fabs(s.u[0][l]), fabs(s.u[0][r])), tmax(fabs(s.u[0][d]), fabs(s.u[0][u])));
  return fabs(s.u[0][me]) + decltype(S0)(2) * S0;
}

// Statistics of row node (j, b): the entropy-bound violation measured as in the node kernel
// (K_i from the stage input of the node and its four neighbours, accurate sigma in float64).
template <int P, int EX, int EY, class LAW, typename T, class S>
__device__ __forceinline__ double line_entropy_violation64(const S& s, int le, int tx, int ty, int j, int b,
                                                           const T* fe, const LawParamsT<T>& lp) {
  using G = LineGeom<P, EX, EY>;
  using N4 = LineNbr<P, EX, EY>;
  constexpr int n = P + 1;
  auto sig = [&](int slot) {
    T uu[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) uu[q] = s.u[q][slot];
    return (double)LAW::rhoe(uu) * (double)powf(uu[0], -lp.gamma);
  };
  const int me = G::rs(le, j) + b;
  double K = sig(me);
  K = fmin(K, sig((b > 0) ? me - 1 : N4::west(le, tx, ty, j)));
  K = fmin(K, sig((b < P) ? me + 1 : N4::east(le, tx, ty, j)));
  K = fmin(K, sig((j > 0) ? G::rs(le, j - 1) + b : N4::south(le, tx, ty, b)));
  K = fmin(K, sig((j < P) ? G::rs(le, j + 1) + b : N4::north(le, tx, ty, b)));
  if (!((double)fe[0] > 0.0)) return 1.0;
  const double sf = (double)LAW::rhoe(fe) * (double)powf(fe[0], -lp.gamma);
  return fmax(0.0, 1.0 - sf / K);
}

// Phase A of the line kernels: the thread's own row (vector loads; slots outside a ragged mesh edge
// hold the boundary ghost of the adjacent element), its per-node quantities (and sigma when SIG) into
// shared memory, then the halo slots.  A thread's first halo slot is loaded before its row is
// processed, so that the two global-load latencies overlap.  The row's state and per-node
// quantities are left in ur and ax.
template <int P, int EX, int EY, class LAW, typename T, bool SIG, class S>
__device__ __forceinline__ void line_phase_a(S& s, const Instance<T>& I, const Tables<T>& tab, const LawParamsT<T>& lp,
                                             int t, bool live, bool act, int j, int ex, int ey, int ex0, int ey0,
                                             long long grow, int srow, T h, T xij, T (&ur)[LAW::NC][P + 1],
                                             typename LAW::Aux (&ax)[P + 1]) {
  using G = LineGeom<P, EX, EY>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const long long N = I.N;
  T uh[NC], hpx = T(0), hpy = T(0);
  const bool h0 = t < G::NH;
  if (h0) halo_load<P, EX, EY, NC>(I, tab, t, ex0, ey0, h, uh, hpx, hpy);
  if (live) {
    if (act) {
#pragma unroll
      for (int q = 0; q < NC; ++q) ld_line<n>(I.uin + q * N + grow, ur[q]);
    } else {
      // slots outside a ragged mesh edge hold the boundary ghost of the adjacent element
#pragma unroll
      for (int b = 0; b < n; ++b) {
        T uu[NC];
        if (ey < I.ny) neighbor_trace<P, NC>(I, 1, I.nx - 1, ey, j, tab.xi, uu);
        else if (ex < I.nx) neighbor_trace<P, NC>(I, 3, ex, I.ny - 1, b, tab.xi, uu);
        else {
#pragma unroll
          for (int q = 0; q < NC; ++q) uu[q] = I.uin[q * N + ((long long)ey0 * I.nx + ex0) * NN];
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) ur[q][b] = uu[q];
      }
    }
    T sg[n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T uu[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) uu[q] = ur[q][b];
      const T px = I.x0 + h * (ex < I.nx ? T(ex) + tab.xi[b] : T(I.nx));
      const T py = I.y0 + h * (ey < I.ny ? T(ey) + xij : T(I.ny));
      node_aux<LAW>(uu, px, py, ax[b], lp);
      sg[b] = (LAW::kEntropy && SIG) ? LAW::sigma(uu, ax[b], lp) : T(0);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) st_line<n>(&s.u[q][srow], ur[q]);
    constexpr int NA = AuxWords<LAW, T>::value;
    if constexpr (NA > 0) {
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        T v[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = reinterpret_cast<const T*>(&ax[b])[k];
        st_line<n>(&s.aux[k][srow], v);
      }
    }
    if constexpr (LAW::kEntropy && SIG) st_line<n>(&s.sig[srow], sg);
  }
  if (h0) {
    typename LAW::Aux ah;
    node_aux<LAW>(uh, hpx, hpy, ah, lp);
    st_node<LAW, T, S, SIG>(s, G::NTP + t, uh, ah, (LAW::kEntropy && SIG) ? LAW::sigma(uh, ah, lp) : T(0));
  }
  for (int hh = t + G::THREADS; hh < G::NH; hh += G::THREADS) {
    T uu[NC], px, py;
    halo_load<P, EX, EY, NC>(I, tab, hh, ex0, ey0, h, uu, px, py);
    typename LAW::Aux ah;
    node_aux<LAW>(uu, px, py, ah, lp);
    st_node<LAW, T, S, SIG>(s, G::NTP + hh, uu, ah, (LAW::kEntropy && SIG) ? LAW::sigma(uu, ah, lp) : T(0));
  }
}

template <int P, int EX, int EY, class LAW, typename T, bool STATS>
__device__ __forceinline__ void stage_lines_body(LineSmem<P, EX, EY, LAW, T>& s, const Instance<T>& I,
                                                 const Tables<T>& tab, const LawParamsT<T>& lp, int tile_x,
                                                 int tile_y) {
  using G = LineGeom<P, EX, EY>;
  using N4 = LineNbr<P, EX, EY>;
  using Nd = LNode<LAW, T>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const int t = threadIdx.x;
  const bool live = (G::NL == G::THREADS) || (t < G::NL);
  const int le = live ? t / n : 0, j = live ? t - le * n : 0;
  const int tx = le % EX, ty = le / EX;
  const int ex0 = tile_x * EX, ey0 = tile_y * EY;
  const int ex = ex0 + tx, ey = ey0 + ty;
  const bool act = live && ex < I.nx && ey < I.ny;
  const long long N = I.N;
  const long long grow = act ? ((long long)ey * I.nx + ex) * NN + j * n : 0;  // global index of node (j, 0)
  const int srow = G::rs(le, j);
  const T h = I.hT;
  const T wj = pick<n>(tab.w, j);
  const T xij = pick<n>(tab.xi, j);

  const T dt = *I.dtT;
  {
    T ur[NC][n];
    typename LAW::Aux ax[n];
    line_phase_a<P, EX, EY, LAW, T, true>(s, I, tab, lp, t, live, act, j, ex, ey, ex0, ey0, grow, srow, h, xij, ur, ax);
  }
  __syncthreads();

  const bool move = (dt > T(0)) && (dt < T(FLT_MAX));

  // ---------------- B: column role (column j of element le)
  if (live) {
    Nd nd[n], lft, rgt;
#pragma unroll
    for (int a = 0; a < n; ++a) ld_node<LAW, T>(s, G::rs(le, a) + j, nd[a]);
    ld_node<LAW, T>(s, N4::south(le, tx, ty, j), lft);
    ld_node<LAW, T>(s, N4::north(le, tx, ty, j), rgt);
    T rl[n][NC], lo[n], hi[n], K[n], S[n][NC];
    line_residuals<P, 1, LAW, T>(tab, lp, nd, lft, rgt, h * wj, rl, lo, hi, K, S);
#pragma unroll
    for (int a = 0; a < n; ++a) {
      const int sl = G::rs(le, a) + j;
#pragma unroll
      for (int q = 0; q < NC; ++q) s.rly[q][sl] = rl[a][q];
      if (a < P) {
#pragma unroll
        for (int q = 0; q < NC; ++q) s.sy[q][sl] = S[a][q];
      }
      s.lo[sl] = lo[a];
      s.hi[sl] = hi[a];
      if constexpr (LAW::kEntropy) s.K[sl] = K[a];
    }
  }

  // ---------------- C: row role (row j of element le)
  T rlx[n][NC], lox[n], hix[n], Kx[n], Sx[n][NC];
  if (live) {
    Nd nd[n], lft, rgt;
    {
      T v[NC][n];
#pragma unroll
      for (int q = 0; q < NC; ++q) ld_line<n>(&s.u[q][srow], v[q]);
#pragma unroll
      for (int b = 0; b < n; ++b)
#pragma unroll
        for (int q = 0; q < NC; ++q) nd[b].u[q] = v[q][b];
      constexpr int NA = AuxWords<LAW, T>::value;
      if constexpr (NA > 0) {
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          T w[n];
          ld_line<n>(&s.aux[k][srow], w);
#pragma unroll
          for (int b = 0; b < n; ++b) reinterpret_cast<T*>(&nd[b].ax)[k] = w[b];
        }
      }
      if constexpr (LAW::kEntropy) {
        T w[n];
        ld_line<n>(&s.sig[srow], w);
#pragma unroll
        for (int b = 0; b < n; ++b) nd[b].s = w[b];
      } else {
#pragma unroll
        for (int b = 0; b < n; ++b) nd[b].s = T(0);
      }
    }
    if constexpr (G::XSHFL) {
      // the row's west neighbour is node P of the same row n lanes down, its east neighbour node 0
      // n lanes up; the tile's edge columns read the halo
      shfl_node<LAW, T>(nd[P], lft, -n);
      shfl_node<LAW, T>(nd[0], rgt, n);
      if (tx == 0) ld_node<LAW, T>(s, G::hW + ty * n + j, lft);
      if (tx == EX - 1) ld_node<LAW, T>(s, G::hE + ty * n + j, rgt);
    } else {
      ld_node<LAW, T>(s, N4::west(le, tx, ty, j), lft);
      ld_node<LAW, T>(s, N4::east(le, tx, ty, j), rgt);
    }
    line_residuals<P, 0, LAW, T>(tab, lp, nd, lft, rgt, h * wj, rlx, lox, hix, Kx, Sx);
  }
  __syncthreads();

  // ---------------- D: per node of the row, u^L, bounds and alpha-tilde
  T uL[n][NC], at[n], dtm[n], lob[n], hib[n];
  T yp[n][NC], ym[n][NC];
  int iters = 0, caps = 0;
  if (live) {
    T u0r[NC][n];
#pragma unroll
    for (int q = 0; q < NC; ++q) ld_line<n>(&s.u[q][srow], u0r[q]);
    T rly[NC][n], lyv[n], hyv[n], kyv[n];
#pragma unroll
    for (int q = 0; q < NC; ++q) ld_line<n>(&s.rly[q][srow], rly[q]);
    ld_line<n>(&s.lo[srow], lyv);
    ld_line<n>(&s.hi[srow], hyv);
    if constexpr (LAW::kEntropy) ld_line<n>(&s.K[srow], kyv);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      T v[n];
      if (j < P) {
        ld_line<n>(&s.sy[q][srow], v);
      } else {
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = T(0);
      }
#pragma unroll
      for (int b = 0; b < n; ++b) yp[b][q] = v[b];
      if (j > 0) {
        ld_line<n>(&s.sy[q][G::rs(le, j > 0 ? j - 1 : 0)], v);
      } else {
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = T(0);
      }
#pragma unroll
      for (int b = 0; b < n; ++b) ym[b][q] = v[b];
    }
    T kb[n];
    unsigned slow = 0;  // nodes whose entropy constraint the cheap certified test leaves undecided
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const T m = h * h * wj * tab.w[b];
      dtm[b] = move ? fdiv(dt, m) : T(0);
      T tq[NC], uu[NC], rr[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) { uu[q] = u0r[q][b]; rr[q] = rly[q][b]; }
      v_add<NC>(tq, rlx[b], rr);
      v_fma<NC>(uL[b], dtm[b], tq, uu);
      const T lo = tmin(lox[b], lyv[b]), hi = tmax(hix[b], hyv[b]);
      lob[b] = lo;
      hib[b] = hi;
      kb[b] = LAW::kEntropy ? tmin(Kx[b], kyv[b]) : T(0);
      T xp[NC], xm[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        xp[q] = (b < P) ? Sx[b][q] : T(0);
        xm[q] = (b > 0) ? Sx[b > 0 ? b - 1 : 0][q] : T(0);
      }
      T a_ = T(1);
      if (move) {
        const T c1 = xp[0], c2 = -xm[0], c3 = yp[b][0], c4 = -ym[b][0];
        const T Pp = tmax(c1, T(0)) + tmax(c2, T(0)) + tmax(c3, T(0)) + tmax(c4, T(0));
        const T Pm = tmin(c1, T(0)) + tmin(c2, T(0)) + tmin(c3, T(0)) + tmin(c4, T(0));
        const T mdt = fdiv(m, dt);
        const T Qp = tmax(T(0), mdt * (hi - uL[b][0]));
        const T Qm = tmin(T(0), mdt * (lo - uL[b][0]));
        const T Rp = (Pp > T(0)) ? tmin(T(1), fdiv(Qp, Pp)) : T(1);
        const T Rm = (Pm < T(0)) ? tmin(T(1), fdiv(Qm, Pm)) : T(1);
        a_ = tmin(Rp, Rm);
        if constexpr (LAW::kEntropy) {
          if (!entropy_certain<LAW>(uL[b], kb[b] * (T(1) + Prec<T>::entropy_margin), xp, xm, yp[b], ym[b],
                                    T(4) * dtm[b], a_, lp))
            slow |= 1u << b;
        }
      }
      at[b] = a_;
    }
    if constexpr (LAW::kEntropy) {
      // the full entropy limiting of the undecided nodes, one node at a time through a single
      // (inlined once) evaluation: the line's values of that node are selected into scalars
#pragma unroll 1
      while (slow) {
        const int bs = __ffs(slow) - 1;
        slow &= slow - 1;
        T u1[NC], xp[NC], xm[NC], y1[NC], y2[NC], K1 = T(0), d1 = T(0), a1 = T(0);
#pragma unroll
        for (int c = 0; c < n; ++c) {
          if (c == bs) {
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              u1[q] = uL[c][q];
              xp[q] = (c < P) ? Sx[c][q] : T(0);
              xm[q] = (c > 0) ? Sx[c > 0 ? c - 1 : 0][q] : T(0);
              y1[q] = yp[c][q];
              y2[q] = ym[c][q];
            }
            K1 = kb[c];
            d1 = dtm[c];
            a1 = at[c];
          }
        }
        const T r = entropy_limit<LAW>(u1, K1 * (T(1) + Prec<T>::entropy_margin), xp, xm, y1, y2, T(4) * d1, a1, lp,
                                       iters, caps);
#pragma unroll
        for (int c = 0; c < n; ++c)
          if (c == bs) at[c] = r;
      }
    }
    if (I.dbg_lo && act) {
#pragma unroll
      for (int b = 0; b < n; ++b) {
        I.dbg_lo[grow + b] = (double)lob[b];
        I.dbg_hi[grow + b] = (double)hib[b];
        I.dbg_K[grow + b] = (double)kb[b];
        I.dbg_alpha[grow + b] = (double)at[b];
      }
    }
    st_line<n>(&s.alpha[srow], at);
  }
  T u0[NC][n];  // u^n for the RK combination; its latency overlaps the barrier
  if (act && I.c0 != T(0)) {
#pragma unroll
    for (int q = 0; q < NC; ++q) ld_line<n>(I.u0 + q * N + grow, u0[q]);
  }
  __syncthreads();

  // ---------------- E: face coefficients, limited update, RK combination
  T vmax = T(0), evmax = T(0);
  int nudged = 0;
  if (live) {
    T aup[n], adn[n];
    if (j < P) ld_line<n>(&s.alpha[G::rs(le, j + 1)], aup);
    if (j > 0) ld_line<n>(&s.alpha[G::rs(le, j - 1)], adn);
    T res[NC][n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const T axp = (b < P) ? tmin(at[b], at[b < P ? b + 1 : b]) : T(0);
      const T axm = (b > 0) ? tmin(at[b], at[b > 0 ? b - 1 : b]) : T(0);
      const T ayp = (j < P) ? tmin(at[b], aup[b]) : T(0);
      const T aym = (j > 0) ? tmin(at[b], adn[b]) : T(0);
      T xp[NC], xm[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        xp[q] = (b < P) ? Sx[b][q] : T(0);
        xm[q] = (b > 0) ? Sx[b > 0 ? b - 1 : 0][q] : T(0);
      }
      T acc[NC], fe[NC];
      v_scale<NC>(acc, axp, xp);
      v_fma<NC>(acc, -axm, xm, acc);
      v_fma<NC>(acc, ayp, yp[b], acc);
      v_fma<NC>(acc, -aym, ym[b], acc);
      v_fma<NC>(fe, dtm[b], acc, uL[b]);
      int nb = 0;
      if constexpr (sizeof(T) == 4) {
        if (!(fe[0] >= lob[b] && fe[0] <= hib[b])) {  // rare: the rounding scale only where it is needed
          const T mag = line_stencil_scale<P, EX, EY>(s, le, tx, ty, j, b) + fabs(uL[b][0]) +
                        tmax(fabs(lob[b]), fabs(hib[b])) +
                        dtm[b] * (fabs(axp * xp[0]) + fabs(axm * xm[0]) + fabs(ayp * yp[b][0]) + fabs(aym * ym[b][0]));
          nb = accept_rounded(fe[0], lob[b], hib[b], mag);
        }
      }
      if constexpr (STATS) {
        if (act && move) {
          const T scale = tmax(tmax(fabs(lob[b]), fabs(hib[b])), T(I.stats->field_scale));
          T v = tmax(lob[b] - fe[0], fe[0] - hib[b]);
          v = (v > T(0)) ? fdiv(v, scale > T(0) ? scale : T(1)) : T(0);
          vmax = tmax(vmax, v);
          if constexpr (LAW::kEntropy) {
            T ev;
            if constexpr (sizeof(T) == 4) {
              ev = T(line_entropy_violation64<P, EX, EY, LAW, T>(s, le, tx, ty, j, b, fe, lp));
            } else {
              // K as the limiter used it: min over the node's four faces
              T kk = tmin(Kx[b], s.K[srow + b]);
              const T sgf = LAW::sigma_of(fe, lp);
              ev = tmax(T(0), T(1) - sgf / kk);
              if (!(fe[0] > T(0))) ev = T(1);
            }
            evmax = tmax(evmax, ev);
          }
        }
        nudged += act ? nb : 0;
      }
      if (I.c0 == T(0)) {
#pragma unroll
        for (int q = 0; q < NC; ++q) res[q][b] = fe[q];
      } else {  // the SSP-RK3 combination c0 u^n + c1 u^FE
        T r1[NC], uu[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) uu[q] = u0[q][b];
        v_scale<NC>(r1, I.c1, fe);
        v_fma<NC>(r1, I.c0, uu, r1);
#pragma unroll
        for (int q = 0; q < NC; ++q) res[q][b] = r1[q];
      }
    }
    if (act) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st_line<n>(I.uout + q * N + grow, res[q]);
    }
  }
  if constexpr (STATS) {
    if (I.stats) {
      warp_rootfind_stats(caps, iters, nudged, I.stats);
      warp_max_atomic(vmax, &I.stats->max_bound_violation);
      warp_max_atomic(evmax, &I.stats->max_entropy_violation);
    }
  }
}

template <int P, int EX, int EY, class LAW, typename T>
struct LineLaunchBounds {
  using G = LineGeom<P, EX, EY>;
  static constexpr int SMEM_CTAS = (int)((227u * 1024u) / (sizeof(LineSmem<P, EX, EY, LAW, T>) + 1024u));
  static constexpr int REG_CTAS = 65536 / (G::THREADS * 128);  // at least 128 registers per thread
  static constexpr int M = SMEM_CTAS < REG_CTAS ? SMEM_CTAS : REG_CTAS;
  static constexpr int MINB = M < 1 ? 1 : M;
};

template <int P, int EX, int EY, class LAW, typename T, bool STATS>
__global__ void __launch_bounds__(LineGeom<P, EX, EY>::THREADS, (LineLaunchBounds<P, EX, EY, LAW, T>::MINB))
k_stage_lines(const StageLaunch<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<LineSmem<P, EX, EY, LAW, T>*>(smem_raw);
  const int tiles_x = (A.inst.nx + EX - 1) / EX;
  const int tile_y = blockIdx.x / tiles_x, tile_x = blockIdx.x - tile_y * tiles_x;
  stage_lines_body<P, EX, EY, LAW, T, STATS>(s, A.inst, A.tab, A.lp, tile_x, tile_y);
}

template <int P, int EX, int EY, class LAW, typename T, bool STATS>
__global__ void __launch_bounds__(LineGeom<P, EX, EY>::THREADS, (LineLaunchBounds<P, EX, EY, LAW, T>::MINB))
k_stage_lines_batch(const BatchLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<LineSmem<P, EX, EY, LAW, T>*>(smem_raw);
  __shared__ Instance<T> sI;
  const int2 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  const int tiles_x = (sI.nx + EX - 1) / EX;
  const int tile_y = task.y / tiles_x, tile_x = task.y - tile_y * tiles_x;
  stage_lines_body<P, EX, EY, LAW, T, STATS>(s, sI, B.tab, B.lp, tile_x, tile_y);
}

template <int P, int EX, int EY, class LAW, typename T, bool STATS>
cudaError_t launch_lines(const StageLaunch<T>& a, cudaStream_t s) {
  using G = LineGeom<P, EX, EY>;
  constexpr size_t smem = sizeof(LineSmem<P, EX, EY, LAW, T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_stage_lines<P, EX, EY, LAW, T, STATS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  const long long tiles = (long long)((a.inst.nx + EX - 1) / EX) * ((a.inst.ny + EY - 1) / EY);
  if (tiles <= 0) return cudaSuccess;
  k_stage_lines<P, EX, EY, LAW, T, STATS><<<(unsigned)tiles, G::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int EX, int EY, class LAW, typename T, bool STATS>
cudaError_t launch_lines_batch(const BatchLaunch<T>& B, cudaStream_t s) {
  using G = LineGeom<P, EX, EY>;
  constexpr size_t smem = sizeof(LineSmem<P, EX, EY, LAW, T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_stage_lines_batch<P, EX, EY, LAW, T, STATS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (B.ntasks <= 0) return cudaSuccess;
  k_stage_lines_batch<P, EX, EY, LAW, T, STATS><<<(unsigned)B.ntasks, G::THREADS, smem, s>>>(B);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- time step (Eq. cfl-low)
// The CFL bound m_i / (2 sum_{j != i} d-hat_ij), d-hat = (h w / 2) lambda on the node's four faces,
// min-reduced into *out_bits, on the line kernel's tiles: each thread evaluates lambda on the faces
// of its row (west/east neighbours as in the stage kernel) and of its column; the column's sums
// reach the row threads through shared memory.  The same face arguments and the same arithmetic as
// the node layout's time-step kernel, hence the same time step.
template <int P, int EX, int EY, class LAW, typename T>
struct LineDtSmem {
  using G = LineGeom<P, EX, EY>;
  static constexpr int NC = LAW::NC, NA = AuxWords<LAW, T>::value;
  T u[NC][G::NS];
  T aux[NA > 0 ? NA : 1][G::NS];
  T ly[G::NTP];  // per node: lambda on its lower plus its upper y face
  T red[32];
};

template <class LAW, typename T, class S>
__device__ __forceinline__ void ld_node_ua(const S& s, int slot, LNode<LAW, T>& nd) {
  constexpr int NA = AuxWords<LAW, T>::value;
#pragma unroll
  for (int q = 0; q < LAW::NC; ++q) nd.u[q] = s.u[q][slot];
  if constexpr (NA > 0) {
    T* aw = reinterpret_cast<T*>(&nd.ax);
#pragma unroll
    for (int k = 0; k < NA; ++k) aw[k] = s.aux[k][slot];
  }
  nd.s = T(0);
}

template <int P, int EX, int EY, class LAW, typename T>
__global__ void __launch_bounds__(LineGeom<P, EX, EY>::THREADS)
k_dt_lines(const StageLaunch<T> A, unsigned long long* out_bits) {
  using G = LineGeom<P, EX, EY>;
  using N4 = LineNbr<P, EX, EY>;
  using Nd = LNode<LAW, T>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<LineDtSmem<P, EX, EY, LAW, T>*>(smem_raw);
  const Instance<T>& I = A.inst;
  const Tables<T>& tab = A.tab;
  const LawParamsT<T>& lp = A.lp;
  const int tiles_x = (I.nx + EX - 1) / EX;
  const int tile_y = blockIdx.x / tiles_x, tile_x = blockIdx.x - tile_y * tiles_x;
  const int t = threadIdx.x;
  const bool live = (G::NL == G::THREADS) || (t < G::NL);
  const int le = live ? t / n : 0, j = live ? t - le * n : 0;
  const int tx = le % EX, ty = le / EX;
  const int ex0 = tile_x * EX, ey0 = tile_y * EY;
  const int ex = ex0 + tx, ey = ey0 + ty;
  const bool act = live && ex < I.nx && ey < I.ny;
  const long long grow = act ? ((long long)ey * I.nx + ex) * NN + j * n : 0;
  const int srow = G::rs(le, j);
  const T h = I.hT;
  const T wj = pick<n>(tab.w, j);
  const T xij = pick<n>(tab.xi, j);
  T ur[NC][n];
  typename LAW::Aux ax[n];
  line_phase_a<P, EX, EY, LAW, T, false>(s, I, tab, lp, t, live, act, j, ex, ey, ex0, ey0, grow, srow, h, xij, ur, ax);
  __syncthreads();
  T lx[n + 1];
  if (live) {
    // column j: lambda on its n + 1 y faces, summed per node for the row threads
    Nd nd[n], lft, rgt;
#pragma unroll
    for (int a = 0; a < n; ++a) ld_node_ua<LAW, T>(s, G::rs(le, a) + j, nd[a]);
    ld_node_ua<LAW, T>(s, N4::south(le, tx, ty, j), lft);
    ld_node_ua<LAW, T>(s, N4::north(le, tx, ty, j), rgt);
    T ly[n + 1];
    ly[0] = LAW::lam(1, lft.u, lft.ax, nd[0].u, nd[0].ax, lp);
#pragma unroll
    for (int a = 1; a < n; ++a) ly[a] = LAW::lam(1, nd[a - 1].u, nd[a - 1].ax, nd[a].u, nd[a].ax, lp);
    ly[n] = LAW::lam(1, nd[P].u, nd[P].ax, rgt.u, rgt.ax, lp);
#pragma unroll
    for (int a = 0; a < n; ++a) s.ly[G::rs(le, a) + j] = ly[a] + ly[a + 1];
    // row j: lambda on its n + 1 x faces
#pragma unroll
    for (int b = 0; b < n; ++b) {
#pragma unroll
      for (int q = 0; q < NC; ++q) nd[b].u[q] = ur[q][b];
      nd[b].ax = ax[b];
      nd[b].s = T(0);
    }
    if constexpr (G::XSHFL) {
      shfl_node<LAW, T>(nd[P], lft, -n);
      shfl_node<LAW, T>(nd[0], rgt, n);
      if (tx == 0) ld_node_ua<LAW, T>(s, G::hW + ty * n + j, lft);
      if (tx == EX - 1) ld_node_ua<LAW, T>(s, G::hE + ty * n + j, rgt);
    } else {
      ld_node_ua<LAW, T>(s, N4::west(le, tx, ty, j), lft);
      ld_node_ua<LAW, T>(s, N4::east(le, tx, ty, j), rgt);
    }
    lx[0] = LAW::lam(0, lft.u, lft.ax, nd[0].u, nd[0].ax, lp);
#pragma unroll
    for (int b = 1; b < n; ++b) lx[b] = LAW::lam(0, nd[b - 1].u, nd[b - 1].ax, nd[b].u, nd[b].ax, lp);
    lx[n] = LAW::lam(0, nd[P].u, nd[P].ax, rgt.u, rgt.ax, lp);
  }
  __syncthreads();
  const T big = T(FLT_MAX);
  T val = big;
  if (act) {
    T lyr[n];
    ld_line<n>(&s.ly[srow], lyr);
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const T wa = wj, wb = tab.w[b];
      const T sumd = T(0.5) * h * wa * (lx[b] + lx[b + 1]) + T(0.5) * h * wb * lyr[b];
      if (sumd > T(0)) val = tmin(val, fdiv(h * h * wa * wb, T(2) * sumd));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val = tmin(val, __shfl_xor_sync(0xffffffffu, val, o));
  if ((t & 31) == 0) s.red[t >> 5] = val;
  __syncthreads();
  if (t < 32) {
    val = (t < G::THREADS / 32) ? s.red[t] : big;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val = tmin(val, __shfl_xor_sync(0xffffffffu, val, o));
    if (t == 0 && val < big) atomicMin(out_bits, (unsigned long long)__double_as_longlong((double)val));
  }
}

template <int P, int EX, int EY, class LAW, typename T>
cudaError_t launch_dt_lines(const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s) {
  using G = LineGeom<P, EX, EY>;
  constexpr size_t smem = sizeof(LineDtSmem<P, EX, EY, LAW, T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_dt_lines<P, EX, EY, LAW, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  const long long tiles = (long long)((a.inst.nx + EX - 1) / EX) * ((a.inst.ny + EY - 1) / EY);
  if (tiles <= 0) return cudaSuccess;
  k_dt_lines<P, EX, EY, LAW, T><<<(unsigned)tiles, G::THREADS, smem, s>>>(a, bits);
  return cudaGetLastError();
}

// Line kernels of one law, degree and precision, by line-tile index: Euler only (the other laws
// have no line-kernel candidates).
template <int LAWID, int P, class LAW, typename T>
struct LineDispatch {
  static cudaError_t stage(int, const StageLaunch<T>&, bool, cudaStream_t) { return cudaErrorInvalidValue; }
  static cudaError_t batch(int, const BatchLaunch<T>&, bool, cudaStream_t) { return cudaErrorInvalidValue; }
  static cudaError_t dt(int, const StageLaunch<T>&, unsigned long long*, cudaStream_t) { return cudaErrorInvalidValue; }
};

template <int P, class LAW, typename T>
struct LineDispatch<LAW_EULER, P, LAW, T> {
  static cudaError_t stage(int lt, const StageLaunch<T>& a, bool stats, cudaStream_t s) {
    constexpr TileShape t0 = kLineTiles[P][0], t1 = kLineTiles[P][1];
    switch (lt) {
      case 0: return stats ? launch_lines<P, t0.tx, t0.ty, LAW, T, true>(a, s) : launch_lines<P, t0.tx, t0.ty, LAW, T, false>(a, s);
      case 1: return stats ? launch_lines<P, t1.tx, t1.ty, LAW, T, true>(a, s) : launch_lines<P, t1.tx, t1.ty, LAW, T, false>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  static cudaError_t dt(int lt, const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s) {
    constexpr TileShape t0 = kLineTiles[P][0], t1 = kLineTiles[P][1];
    switch (lt) {
      case 0: return launch_dt_lines<P, t0.tx, t0.ty, LAW, T>(a, bits, s);
      case 1: return launch_dt_lines<P, t1.tx, t1.ty, LAW, T>(a, bits, s);
      default: return cudaErrorInvalidValue;
    }
  }
  static cudaError_t batch(int lt, const BatchLaunch<T>& b, bool stats, cudaStream_t s) {
    constexpr TileShape t0 = kLineTiles[P][0], t1 = kLineTiles[P][1];
    switch (lt) {
      case 0: return stats ? launch_lines_batch<P, t0.tx, t0.ty, LAW, T, true>(b, s) : launch_lines_batch<P, t0.tx, t0.ty, LAW, T, false>(b, s);
      case 1: return stats ? launch_lines_batch<P, t1.tx, t1.ty, LAW, T, true>(b, s) : launch_lines_batch<P, t1.tx, t1.ty, LAW, T, false>(b, s);
      default: return cudaErrorInvalidValue;
    }
  }
};

}  // namespace sidp
