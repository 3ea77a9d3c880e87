// Stage and time-step kernels on curved (mapped) quadrilateral meshes (Sec. 2.3, Sec. 3.1, with
// the limiting of Sec. 4 and the CFL bound of Eq. cfl-low).
//
// Per-node geometry (float64 on the host, converted to the stage precision), kGeoFields arrays of
// N values: rows 1 and 2 of G J^-1 (x, y components), the corrected rows of Sec. 3.1, the mass
// m_i = w_a w_b G_i, and the face normals (+xi at b = 0, p; +eta at a = 0, p; one value per face,
// shared by the two elements of the face).
//
// One CTA holds EPB whole elements, one thread per node.  Every face of an element is evaluated
// inside it: the element faces from the node's own state and the neighbour's trace (read from
// global memory, the L2-resident neighbour), the internal subcell faces between neighbouring
// nodes of a line from shared memory.  Two elements that share a face evaluate its flux from the
// same operands in the same order (the -xi/-eta side as the left state), so the update is
// conservative.
//
// On a mapped element the pair coefficients are c_ij = D-hat^T_ij (row-hat)_j (the metric at node
// j).  Along a line, with the contravariant low-order flux g = row-hat . F at each node, the
// pairwise form of Eq. dg-lo-cij becomes a difference of subcell fluxes
//   G_{b+1/2} = (g_b + g_{b+1})/2 - Lambda/2 (u_{b+1} - u_b),
//   Lambda = max(lambda(u_b, u_{b+1}, row_{b+1}) |row_{b+1}|, lambda(u_b, u_{b+1}, row_b) |row_b|),
// d_ij = w Lambda / 2 (Eq. dij with n_ij = -c_ij/|c_ij|), and the two nodes of a subcell face
// have the bar states u-bar = (u_b + u_{b+1})/2 - row_other . (F_{b+1} - F_b) / (2 Lambda)
// (Eq. bar-states with c_ij != -c_ji).
//
// Limiters: none, low-order, subcell (Sec. 4.1.3, 4.3) and, as a compile-time variant, elementwise
// (Sec. 4.1.2, 4.2.1); the smoothness indicator of Sec. 4.4 relaxes the bounds when it is on (its
// modal expansion taken on the reference element).
#pragma once
#include "sidp_kernels.cuh"

namespace sidp {

enum GeoField { GEO_R1X, GEO_R1Y, GEO_R2X, GEO_R2Y, GEO_Q1X, GEO_Q1Y, GEO_Q2X, GEO_Q2Y, GEO_MASS,
                GEO_NXX, GEO_NXY, GEO_NYX, GEO_NYY };
static_assert(GEO_NYY + 1 == kGeoFields, "geometry layout");
static_assert(GEO_MASS == GEO_MASS_FIELD, "geometry layout");

template <int P>
struct CurvedGeom {
  static constexpr int n = P + 1, NN = n * n;
  static constexpr int EPB = (256 / NN) > 0 ? 256 / NN : 1;  // elements per CTA
  static constexpr int THREADS = EPB * NN;                    // 245..256: every thread owns a node
  static_assert(THREADS >= 32 && THREADS <= 256, "block shape");
};

// Resident CTAs per SM the register budget is sized for: float32 kernels take 4 (64 registers,
// a few dozen bytes spilled at p = 3; measured faster than 3 CTAs at 80 registers without
// spills); the float64 ones need more registers than 2 CTAs allow without spilling.
template <typename T> struct CurvedMinBlocks { static constexpr int value = sizeof(T) == 4 ? 4 : 1; };

// One element face as seen from one of its nodes: the face flux, the node's own F . n (the
// high-order face term), the bar state of the limited field, sigma of the neighbour's trace,
// lambda |n| (time step) and |u| of the neighbour's trace (operand scale of the face).  dir 0:
// x face (b = 0 or p), dir 1: y face (a = 0 or p).
template <int P, class LAW, typename T>
struct CurvedFace {
  T Fh[LAW::NC];   // flux in +xi (+eta)
  T Fn[LAW::NC];   // own F . n
  T bar, sig, ln;
  T um;
};

template <int P, class LAW, typename T>
struct CurvedSmem {
  static constexpr int NC = LAW::NC, TH = CurvedGeom<P>::THREADS;
  Vec<T, NC> u[TH];
  typename LAW::Aux aux[TH];
  Vec<T, NC> f1[TH], f2[TH];  // high-order contravariant fluxes (G J^-1 row k) . F
  Vec<T, NC> g1[TH], g2[TH];  // low-order contravariant fluxes (corrected rows)
  Vec<T, NC> Gx[TH], Gy[TH];  // subcell-face fluxes at (a, b+1/2), (a+1/2, b); then r_x, r_y
  T q[TH][4];                 // corrected rows: row 1 (x, y), row 2 (x, y)
  T F0[TH][2];                // x and y fluxes of the limited field
  T bar[TH][4];               // limited-field bar states: x face (left node, right node), y face (lower, upper)
  T lam[TH][2];               // Lambda of the x and y subcell faces (time step)
  T sig[TH];
  T alpha[TH];
  T aK[CurvedGeom<P>::EPB];   // elementwise limiting: alpha_K per element
  T eps[CurvedGeom<P>::EPB];  // smoothness indicator: epsilon_K per element
  CurvedFace<P, LAW, T> cy[CurvedGeom<P>::EPB][4];  // the corners' y faces, evaluated by interior nodes
};

// Element-face neighbour of node (a, b) of element e on side s (0 W, 1 E, 2 S, 3 N): the global
// index of the neighbour's node at the same point, or -1 at a non-periodic boundary (outflow:
// the node's own trace).
template <int P>
__device__ __forceinline__ long long curved_nbr(const int* bc, int nx, int ny, long long e, int a, int b, int s) {
  constexpr int n = P + 1, NN = n * n;
  const int ei = (int)e;  // element indices fit in int (a mesh has fewer than 2^31 elements)
  int ey = ei / nx, ex = ei - ey * nx;
  int na = a, nb = b;
  if (s == 0) { if (ex == 0 && bc[0] != SIDP_BC_PERIODIC) return -1; ex = (ex == 0) ? nx - 1 : ex - 1; nb = P; }
  else if (s == 1) { if (ex == nx - 1 && bc[1] != SIDP_BC_PERIODIC) return -1; ex = (ex == nx - 1) ? 0 : ex + 1; nb = 0; }
  else if (s == 2) { if (ey == 0 && bc[2] != SIDP_BC_PERIODIC) return -1; ey = (ey == 0) ? ny - 1 : ey - 1; na = P; }
  else { if (ey == ny - 1 && bc[3] != SIDP_BC_PERIODIC) return -1; ey = (ey == ny - 1) ? 0 : ey + 1; na = 0; }
  return ((long long)ey * nx + ex) * NN + na * n + nb;
}

// Element-face work of a thread.  An element has 4 (p+1) (node, direction) face evaluations: one
// for each edge node and two for each corner.  Each edge node and each corner's x face is
// evaluated by the node itself, each corner's y face by one of the first four interior nodes
// (p >= 3; for p < 3, where there are too few, by the corner in a second pass).  Every thread
// then runs one evaluation of the same code (no branch per direction or side), and its loads
// of the neighbour's trace and of the face normal are issued with the node's own loads.
template <int P>
struct FaceItem {
  int a, b, dir, side;
  int corner;  // an interior node's corner (0..3: (0,0), (0,p), (p,0), (p,p)), else -1
  bool on;
};

template <int P>
__device__ __forceinline__ FaceItem<P> face_item(int a, int b, bool act) {
  FaceItem<P> it{a, b, 0, 0, -1, act};
  if (b == 0 || b == P) {
    it.dir = 0;
  } else if (a == 0 || a == P) {
    it.dir = 1;
  } else {
    const int k = (a - 1) * (P - 1) + (b - 1);
    if (k < 4) {
      it.a = (k >> 1) ? P : 0;
      it.b = (k & 1) ? P : 0;
      it.dir = 1;
      it.corner = k;
    } else {
      it.on = false;
    }
  }
  it.side = 2 * it.dir + (((it.dir == 0) ? it.b : it.a) == 0 ? 0 : 1);
  return it;
}

// Global loads of a face evaluation: the face normal of the item's node and, across a shared face,
// the neighbour's trace (ext false at an outflow or wall side: the ghost is built from the own
// trace once it is in shared memory).
template <int P, class LAW, typename T>
__device__ __forceinline__ void face_prefetch(const Instance<T>& I, long long e, const FaceItem<P>& it, T* un,
                                              T& nvx, T& nvy, bool& ext) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const long long N = I.N, gi = e * NN + it.a * n + it.b;
  nvx = I.geo[(it.dir == 0 ? GEO_NXX : GEO_NYX) * N + gi];
  nvy = I.geo[(it.dir == 0 ? GEO_NXY : GEO_NYY) * N + gi];
  const long long gn = curved_nbr<P>(I.bc, I.nx, I.ny, e, it.a, it.b, it.side);
  ext = gn >= 0;
#pragma unroll
  for (int q = 0; q < NC; ++q) un[q] = ext ? I.uin[q * N + gn] : T(0);
}

// One face evaluation (after the node states are in shared memory): the ghost at a boundary
// (outflow: the own trace; slip wall, Sec. 5.7: the own trace with its momentum reflected about
// the face's unit normal, m - 2 (m . n) n), then the flux with the -xi/-eta side as the left state.
template <int P, class LAW, typename T>
__device__ __forceinline__ void face_eval(const CurvedSmem<P, LAW, T>& s, const Instance<T>& I,
                                          const LawParamsT<T>& lp, const FaceItem<P>& it, int le, T* un, T nvx,
                                          T nvy, bool ext, CurvedFace<P, LAW, T>& F) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  using Aux = typename LAW::Aux;
  const int slot = le * NN + it.a * n + it.b;
  const Vec<T, NC> uo = s.u[slot];
  const Aux ao = s.aux[slot];
  if (!ext) {
#pragma unroll
    for (int q = 0; q < NC; ++q) un[q] = uo.v[q];
    if constexpr (NC == 4) {
      if (I.bc[it.side] == SIDP_BC_SLIP_WALL) {
        const T inn = frcp(psqrt(nvx * nvx + nvy * nvy));
        const T nx = nvx * inn, ny = nvy * inn;
        const T mn = uo.v[1] * nx + uo.v[2] * ny;
        un[1] = uo.v[1] - T(2) * mn * nx;
        un[2] = uo.v[2] - T(2) * mn * ny;
      }
    }
  }
  Aux an;
  LAW::aux(un, an, lp);
  // operands ordered by selects, not by a branch per side
  const bool low = (it.side & 1) == 0;  // the neighbour is the left state
  T uL[NC], uR[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    uL[q] = low ? un[q] : uo.v[q];
    uR[q] = low ? uo.v[q] : un[q];
  }
  const Aux aL = low ? an : ao, aR = low ? ao : an;
  T fLx[NC], fLy[NC], fRx[NC], fRy[NC];
  LAW::flux(uL, aL, 0, fLx, lp);
  LAW::flux(uL, aL, 1, fLy, lp);
  LAW::flux(uR, aR, 0, fRx, lp);
  LAW::flux(uR, aR, 1, fRy, lp);
  const T nn = psqrt(nvx * nvx + nvy * nvy);
  const T lam = LAW::lam_n(uL, aL, uR, aR, fdiv(nvx, nn), fdiv(nvy, nn), lp);
  F.ln = lam * nn;
  {
    T sx[NC], sy[NC], du[NC], ox[NC], oy[NC];
    v_add<NC>(sx, fLx, fRx);
    v_add<NC>(sy, fLy, fRy);
    v_scale<NC>(sx, nvx, sx);
    v_fma<NC>(sx, nvy, sy, sx);  // (F_L + F_R) . n
    v_scale<NC>(sx, T(0.5), sx);
    v_sub<NC>(du, uR, uL);
    v_fma<NC>(F.Fh, T(-0.5) * F.ln, du, sx);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      ox[q] = low ? fRx[q] : fLx[q];
      oy[q] = low ? fRy[q] : fLy[q];
    }
    v_scale<NC>(F.Fn, nvx, ox);
    v_fma<NC>(F.Fn, nvy, oy, F.Fn);
  }
  const T dF = (fRx[0] - fLx[0]) * nvx + (fRy[0] - fLy[0]) * nvy;
  F.bar = T(0.5) * (uL[0] + uR[0]) - ((F.ln > T(0)) ? fdiv(dF, T(2) * F.ln) : T(0));
  if constexpr (LAW::kEntropy) F.sig = LAW::sigma(un, an, lp);
  else F.sig = T(0);
  F.um = fabs(un[0]);
}

// Operand scale of the low-order state of node (a, b) in slot t (the limited field): |u_i| +
// 2 max |u_j| over its four neighbours (within the element from shared memory; across an element
// face the neighbour's trace, um), as in the Cartesian kernel's stencil_scale.
template <int P, class S, typename T>
__device__ __forceinline__ T curved_stencil_scale(const S& s, int t, int a, int b, T u0, T umx, T umy) {
  constexpr int n = P + 1;
  const T sl = (b > 0) ? fabs(s.u[t - 1].v[0]) : umx, sr = (b < P) ? fabs(s.u[t + 1].v[0]) : umx;
  const T sd = (a > 0) ? fabs(s.u[t - n].v[0]) : umy, su = (a < P) ? fabs(s.u[t + n].v[0]) : umy;
  return fabs(u0) + T(2) * tmax(tmax(sl, sr), tmax(sd, su));
}

// Internal subcell face between slots L and R (dir 0: x, row 1; dir 1: y, row 2).
template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_internal_face(CurvedSmem<P, LAW, T>& s, int L, int R, int dir,
                                                     const LawParamsT<T>& lp) {
  constexpr int NC = LAW::NC;
  const Vec<T, NC> uL = s.u[L], uR = s.u[R];
  const typename LAW::Aux aL = s.aux[L], aR = s.aux[R];
  const int k = 2 * dir;
  const T qLx = s.q[L][k], qLy = s.q[L][k + 1], qRx = s.q[R][k], qRy = s.q[R][k + 1];
  const T nL = psqrt(qLx * qLx + qLy * qLy), nR = psqrt(qRx * qRx + qRy * qRy);
  const T lR = LAW::lam_n(uL.v, aL, uR.v, aR, fdiv(qRx, nR), fdiv(qRy, nR), lp) * nR;
  const T lL = LAW::lam_n(uL.v, aL, uR.v, aR, fdiv(qLx, nL), fdiv(qLy, nL), lp) * nL;
  const T Lam = tmax(lR, lL);
  const Vec<T, NC> gL = dir == 0 ? s.g1[L] : s.g2[L], gR = dir == 0 ? s.g1[R] : s.g2[R];
  Vec<T, NC> G, gs, du;
  v_add<NC>(gs.v, gL.v, gR.v);
  v_sub<NC>(du.v, uR.v, uL.v);
  v_scale<NC>(gs.v, T(0.5), gs.v);
  v_fma<NC>(G.v, T(-0.5) * Lam, du.v, gs.v);
  const T dFx = s.F0[R][0] - s.F0[L][0], dFy = s.F0[R][1] - s.F0[L][1];
  const T mid = T(0.5) * (uL.v[0] + uR.v[0]);
  const T inv2 = (Lam > T(0)) ? fdiv(T(1), T(2) * Lam) : T(0);
  if (dir == 0) s.Gx[L] = G; else s.Gy[L] = G;
  s.bar[L][k] = mid - (qRx * dFx + qRy * dFy) * inv2;      // for the left / lower node
  s.bar[L][k + 1] = mid - (qLx * dFx + qLy * dFy) * inv2;  // for the right / upper node
  s.lam[L][dir] = Lam;
}

// Phase A and the subcell faces, shared by the stage and the time-step kernels.  Returns the
// node's own state, aux, fluxes and its element faces.
template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_load(CurvedSmem<P, LAW, T>& s, const Instance<T>& I, const LawParamsT<T>& lp,
                                            long long e, bool act, int t, int a, int b, T* u, typename LAW::Aux& ax,
                                            CurvedFace<P, LAW, T>& FX, CurvedFace<P, LAW, T>& FY, bool& onx, bool& ony) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const long long N = I.N, g = act ? e * NN + a * n + b : 0;
  const T* geo = I.geo;
  // this thread's element-face evaluation: its global loads go out with the node's own
  const FaceItem<P> it = face_item<P>(a, b, act);
  T un[NC], nvx = T(0), nvy = T(0);
  bool ext = false;
  if (it.on) face_prefetch<P, LAW>(I, e, it, un, nvx, nvy, ext);
#pragma unroll
  for (int q = 0; q < NC; ++q) u[q] = I.uin[q * N + g];
  LAW::aux(u, ax, lp);
  T fx[NC], fy[NC];
  LAW::flux(u, ax, 0, fx, lp);
  LAW::flux(u, ax, 1, fy, lp);
  const T r1x = geo[GEO_R1X * N + g], r1y = geo[GEO_R1Y * N + g], r2x = geo[GEO_R2X * N + g], r2y = geo[GEO_R2Y * N + g];
  const T q1x = geo[GEO_Q1X * N + g], q1y = geo[GEO_Q1Y * N + g], q2x = geo[GEO_Q2X * N + g], q2y = geo[GEO_Q2Y * N + g];
  Vec<T, NC> vu, f1, f2, g1, g2;
#pragma unroll
  for (int q = 0; q < NC; ++q) vu.v[q] = u[q];
  v_scale<NC>(f1.v, r1y, fy);
  v_fma<NC>(f1.v, r1x, fx, f1.v);
  v_scale<NC>(f2.v, r2y, fy);
  v_fma<NC>(f2.v, r2x, fx, f2.v);
  v_scale<NC>(g1.v, q1y, fy);
  v_fma<NC>(g1.v, q1x, fx, g1.v);
  v_scale<NC>(g2.v, q2y, fy);
  v_fma<NC>(g2.v, q2x, fx, g2.v);
  s.u[t] = vu;
  s.aux[t] = ax;
  s.f1[t] = f1;
  s.f2[t] = f2;
  s.g1[t] = g1;
  s.g2[t] = g2;
  s.q[t][0] = q1x; s.q[t][1] = q1y; s.q[t][2] = q2x; s.q[t][3] = q2y;
  s.F0[t][0] = fx[0];
  s.F0[t][1] = fy[0];
  if constexpr (LAW::kEntropy) s.sig[t] = LAW::sigma(u, ax, lp);
  else s.sig[t] = T(0);
  onx = act && (b == 0 || b == P);
  ony = act && (a == 0 || a == P);
  const int le = t / NN;
  __syncthreads();
  // subcell faces as one list over the CTA, all x faces (b < p) and then all y faces (a < p): the
  // last round leaves whole warps idle instead of every warp running both directions
  {
    constexpr int FPE = P * n;                        // faces per element and direction
    constexpr int NXF = CurvedGeom<P>::EPB * FPE;     // x faces of the CTA
#pragma unroll
    for (int f = t; f < 2 * NXF; f += CurvedGeom<P>::THREADS) {
      const int dir = f >= NXF ? 1 : 0;
      const int r = f - dir * NXF;
      const int fe = r / FPE, j = r - fe * FPE;
      const int L = fe * NN + (dir ? j : (j / P) * n + j % P);
      curved_internal_face<P, LAW>(s, L, L + (dir ? n : 1), dir, lp);
    }
  }
  CurvedFace<P, LAW, T> R{};
  if (it.on) face_eval<P, LAW>(s, I, lp, it, le, un, nvx, nvy, ext, R);
  if (it.corner >= 0) s.cy[le][it.corner] = R;
  FX = R;  // the node's own item is its x face wherever it has one (edges W/E and corners)
  FY = R;  // and its y face on the S/N edges; corners take theirs below
  const int k = (a == P ? 2 : 0) + (b == P ? 1 : 0);  // corner index, when onx && ony
  constexpr int kHelped = (P - 1) * (P - 1) < 4 ? (P - 1) * (P - 1) : 4;  // corners with a helper
  if constexpr (kHelped < 4) {
    // p < 3: too few interior nodes; the remaining corners evaluate their y face themselves
    if (onx && ony && k >= kHelped) {
      const FaceItem<P> iy{a, b, 1, 2 + (a == 0 ? 0 : 1), -1, true};
      T un2[NC], nx2, ny2;
      bool ext2;
      face_prefetch<P, LAW>(I, e, iy, un2, nx2, ny2, ext2);
      face_eval<P, LAW>(s, I, lp, iy, le, un2, nx2, ny2, ext2, FY);
    }
  }
  __syncthreads();
  if (onx && ony && k < kHelped) FY = s.cy[le][k];
}


// Entropy-bound violation of a limited float32 result fe at node (a, b) of element e, slot t:
// max(0, 1 - sigma(fe) / K_i) with K_i = min sigma over the node and its four neighbours of the
// stage input, sigma evaluated accurately (compensated rho e, the ratio in float64) as in the
// Cartesian statistics.  In-element neighbours come from shared memory, the neighbour across an
// element face from global memory; an outflow or slip-wall ghost has the node's own sigma (the
// mirrored momentum keeps |m|).  Statistics kernels only.
template <int P, class LAW, typename T>
__device__ double curved_entropy_violation64(const CurvedSmem<P, LAW, T>& s, const Instance<T>& I,
                                             const LawParamsT<T>& lp, long long e, int t, int a, int b,
                                             const T* fe) {
  constexpr int n = P + 1, NC = LAW::NC;
  auto sig = [&](const T* u) { return (double)LAW::rhoe(u) * (double)powf(u[0], -lp.gamma); };
  double K = sig(s.u[t].v);
  if (b > 0) K = fmin(K, sig(s.u[t - 1].v));
  if (b < P) K = fmin(K, sig(s.u[t + 1].v));
  if (a > 0) K = fmin(K, sig(s.u[t - n].v));
  if (a < P) K = fmin(K, sig(s.u[t + n].v));
  const int sides[2] = {b == 0 ? 0 : (b == P ? 1 : -1), a == 0 ? 2 : (a == P ? 3 : -1)};
  for (int k = 0; k < 2; ++k) {
    if (sides[k] < 0) continue;
    const long long gn = curved_nbr<P>(I.bc, I.nx, I.ny, e, a, b, sides[k]);
    if (gn < 0) continue;
    T un[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) un[q] = I.uin[q * I.N + gn];
    K = fmin(K, sig(un));
  }
  if (!((double)fe[0] > 0.0)) return 1.0;
  return fmax(0.0, 1.0 - sig(fe) / K);
}

// Bound and entropy violations of one limited result (statistics kernels only), as in the
// Cartesian stage statistics: the excess over [lo, hi] relative to max(|bound|, field scale), and
// max(0, 1 - sigma(fe)/K).
template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_violations(const CurvedSmem<P, LAW, T>& s, const Instance<T>& I,
                                                  const LawParamsT<T>& lp, long long e, int t, int a, int b,
                                                  const T* fe, T lo, T hi, T K, T& v, T& ev) {
  const T scale = tmax(tmax(fabs(lo), fabs(hi)), T(I.stats->field_scale));
  v = tmax(lo - fe[0], fe[0] - hi);
  v = (v > T(0)) ? fdiv(v, scale > T(0) ? scale : T(1)) : T(0);
  ev = T(0);
  if constexpr (LAW::kEntropy) {
    if constexpr (sizeof(T) == 4) {
      ev = T(curved_entropy_violation64<P, LAW, T>(s, I, lp, e, t, a, b, fe));
    } else {
      ev = tmax(T(0), T(1) - LAW::sigma_of(fe, lp) / K);
      if (!(fe[0] > T(0))) ev = T(1);
    }
  }
}

// Stage statistics of a curved CTA (all threads call it; statistics kernels only).  The CTA need
// not be a whole number of warps, so the per-node values go through shared memory (the rows and
// fluxes of phase B, read for the last time before phase C) and the first, always complete, warp
// reduces them: one atomic per CTA and quantity.
template <int P, class LAW, typename T>
__device__ void curved_stats(CurvedSmem<P, LAW, T>& s, StageStats* st, T v, T ev, int caps, int iters, int nudged) {
  constexpr int TH = CurvedGeom<P>::THREADS;
  const int t = threadIdx.x;
  s.q[t][0] = v;
  s.q[t][1] = ev;
  s.q[t][2] = T(caps);
  s.q[t][3] = T(iters);
  s.F0[t][0] = T(nudged);
  __syncthreads();
  if (t < 32) {
    double mv = 0.0, me = 0.0;
    int c = 0, m = 0, gs = 0;
    for (int j = t; j < TH; j += 32) {
      mv = fmax(mv, (double)s.q[j][0]);
      me = fmax(me, (double)s.q[j][1]);
      c += (int)s.q[j][2];
      m = max(m, (int)s.q[j][3]);
      gs += (int)s.F0[j][0];
    }
    warp_rootfind_stats(c, m, gs, st);
    warp_max_atomic(mv, &st->max_bound_violation);
    warp_max_atomic(me, &st->max_entropy_violation);
  }
}

}  // namespace sidp

namespace sidp {

// One stage on element block eb (elements eb * EPB ...) of instance I.  ELW: elementwise limiting
// (Sec. 4.1.2, 4.2.1) instead of the subcell limiter.  STATS: the variant with the per-stage
// statistics (launched when they are on).
template <int P, class LAW, typename T, bool ELW, bool STATS>
__device__ __forceinline__ void curved_stage_body(CurvedSmem<P, LAW, T>& s, const Instance<T>& I, const Tables<T>& tab,
                                                  const LawParamsT<T>& lp, const SmoothnessT<T>& si, int limiter,
                                                  long long eb) {
  using Gm = CurvedGeom<P>;
  using V = Vec<T, LAW::NC>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const int t = threadIdx.x, le = t / NN, i = t - le * NN, a = i / n, b = i - a * n;
  const long long e = eb * Gm::EPB + le;
  const bool act = e < (long long)I.nx * I.ny;
  const long long N = I.N, g = act ? e * NN + i : 0;

  // ---------------- A, B: node data, element faces, subcell faces
  T u[NC];
  typename LAW::Aux ax;
  CurvedFace<P, LAW, T> FX{}, FY{};
  bool onx, ony;
  curved_load<P, LAW>(s, I, lp, e, act, t, a, b, u, ax, FX, FY, onx, ony);

  // ---------------- smoothness indicator (Sec. 4.4) on the reference element: Legendre
  // coefficients of the limited field (separable nodal -> modal transform), s_K =
  // log10(||u - u-hat||^2 / ||u||^2) with u-hat dropping the modes of degree p in either variable
  if (si.on && limiter >= 2) {
    const int base = le * NN;
    T c1 = T(0);
#pragma unroll
    for (int c = 0; c < n; ++c) c1 += tab.Vinv[b * n + c] * s.u[base + a * n + c].v[0];
    s.alpha[t] = c1;
    __syncthreads();
    T cc = T(0);
#pragma unroll
    for (int c = 0; c < n; ++c) cc += tab.Vinv[a * n + c] * s.alpha[base + c * n + b];
    const T wgt = cc * cc * tab.nrm[a] * tab.nrm[b];
    __syncthreads();
    s.alpha[t] = wgt;
    __syncthreads();
    if (i == 0) {
      T tot = T(0), top = T(0);
      for (int j = 0; j < NN; ++j) {
        const T v = s.alpha[base + j];
        tot += v;
        if (j / n == P || j % n == P) top += v;
      }
      T ek = T(0);
      if (tot > T(0) && top > T(0)) {
        const T sk = plog10(top / tot);
        ek = (sk < si.s0 - si.kappa) ? T(0)
           : (sk > si.s0 + si.kappa) ? T(1)
           : T(0.5) + T(0.5) * psin(T(3.14159265358979323846) * (sk - si.s0) / (T(2) * si.kappa));
      }
      s.eps[le] = ek;
    }
    __syncthreads();
  }

  // ---------------- C: residuals, low-order state, bounds
  const T dt = *I.dtT;
  const bool move = (dt > T(0)) && (dt < T(FLT_MAX));
  const T wa = tab.w[a], wb = tab.w[b];
  const T m = I.geo[GEO_MASS * N + g];
  const T dtm = move ? fdiv(dt, m) : T(0);
  T sx[NC], sy[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) { sx[q] = T(0); sy[q] = T(0); }
  const int lx = le * NN + a * n, ly = le * NN + b;
#pragma unroll
  for (int c = 0; c < n; ++c) {
    const V F1c = s.f1[lx + c], F2c = s.f2[ly + c * n];
    const T dx = tab.D[b * n + c], dy = tab.D[a * n + c];
    v_fma<NC>(sx, dx, F1c.v, sx);
    v_fma<NC>(sy, dy, F2c.v, sy);
  }
  const V Gr = (b < P) ? s.Gx[t] : V{}, Gl = (b > 0) ? s.Gx[t - 1] : V{};
  const V Gu = (a < P) ? s.Gy[t] : V{}, Gd = (a > 0) ? s.Gy[t - n] : V{};
  T uL[NC], rx[NC], ry[NC], out[NC];
  T gr[NC], gl[NC], gu[NC], gd[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    if (b == 0) sx[q] += FX.Fn[q] - FX.Fh[q];
    if (b == P) sx[q] += FX.Fh[q] - FX.Fn[q];
    if (a == 0) sy[q] += FY.Fn[q] - FY.Fh[q];
    if (a == P) sy[q] += FY.Fh[q] - FY.Fn[q];
    gr[q] = (b < P) ? Gr.v[q] : FX.Fh[q];
    gl[q] = (b > 0) ? Gl.v[q] : FX.Fh[q];
    gu[q] = (a < P) ? Gu.v[q] : FY.Fh[q];
    gd[q] = (a > 0) ? Gd.v[q] : FY.Fh[q];
  }
  {
    T rHx[NC], rHy[NC], rLx[NC], rLy[NC], tq[NC];
    v_scale<NC>(rHx, -wa, sx);
    v_scale<NC>(rHy, -wb, sy);
    v_sub<NC>(tq, gr, gl);
    v_scale<NC>(rLx, -wa, tq);
    v_sub<NC>(tq, gu, gd);
    v_scale<NC>(rLy, -wb, tq);
    v_add<NC>(tq, rLx, rLy);
    v_fma<NC>(uL, dtm, tq, u);
    if (limiter == 0) {
      v_add<NC>(tq, rHx, rHy);
      v_fma<NC>(out, dtm, tq, u);
    } else {
#pragma unroll
      for (int q = 0; q < NC; ++q) out[q] = uL[q];
    }
    v_sub<NC>(rx, rHx, rLx);
    v_sub<NC>(ry, rHy, rLy);
  }
  if (limiter < 2 && act) {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      I.uout[q * N + g] = (I.c0 == T(0)) ? out[q] : I.c0 * I.u0[q * N + g] + I.c1 * out[q];
  }
  if (limiter < 2) return;  // uniform across the CTA
  const T bl = (b > 0) ? s.bar[t - 1][1] : FX.bar, br = (b < P) ? s.bar[t][0] : FX.bar;
  const T bd = (a > 0) ? s.bar[t - n][3] : FY.bar, bu = (a < P) ? s.bar[t][2] : FY.bar;
  T lo = tmin(tmin(u[0], tmin(bl, br)), tmin(bd, bu));
  T hi = tmax(tmax(u[0], tmax(bl, br)), tmax(bd, bu));
  if (si.on) {  // Eq. relaxed-bounds
    const T ek = s.eps[le];
    lo = ek * lo + (T(1) - ek) * si.gmin;
    hi = ek * hi + (T(1) - ek) * si.gmax;
  }
  T K = T(0);
  if constexpr (LAW::kEntropy) {
    const T sl = (b > 0) ? s.sig[t - 1] : FX.sig, sr = (b < P) ? s.sig[t + 1] : FX.sig;
    const T sd = (a > 0) ? s.sig[t - n] : FY.sig, su = (a < P) ? s.sig[t + n] : FY.sig;
    K = tmin(tmin(s.sig[t], tmin(sl, sr)), tmin(sd, su));
  }
  if constexpr (ELW) {
    // ---------------- elementwise: alpha-tilde_i for the nodal flux r_i = r_x + r_y, alpha_K = min
    T rn[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) rn[q] = rx[q] + ry[q];
    T at = T(1);
    int iters = 0, caps = 0;
    if (act && move) {
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
    s.alpha[t] = at;
    if (I.dbg_lo && act) {
      I.dbg_lo[g] = (double)lo;
      I.dbg_hi[g] = (double)hi;
      I.dbg_K[g] = (double)K;
      I.dbg_alpha[g] = (double)at;
    }
    __syncthreads();
    if (i == 0) {
      T mn = T(1);
      for (int j = 0; j < NN; ++j) mn = tmin(mn, s.alpha[le * NN + j]);
      s.aK[le] = mn;
    }
    __syncthreads();
    T v = T(0), ev = T(0);
    int nudged = 0;
    if (act) {
      const T ak = s.aK[le];
      T fe[NC];
      v_fma<NC>(fe, ak * dtm, rn, uL);
      if constexpr (sizeof(T) == 4) {
        if (!(fe[0] >= lo && fe[0] <= hi))  // rare: the rounding scale only where it is needed
          nudged = accept_rounded(fe[0], lo, hi, curved_stencil_scale<P>(s, t, a, b, u[0], FX.um, FY.um) +
                                                     fabs(uL[0]) + fabs(ak * dtm * rn[0]) + tmax(fabs(lo), fabs(hi)));
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) I.uout[q * N + g] = (I.c0 == T(0)) ? fe[q] : I.c0 * I.u0[q * N + g] + I.c1 * fe[q];
      if constexpr (STATS) {
        if (I.stats && move) curved_violations<P, LAW, T>(s, I, lp, e, t, a, b, fe, lo, hi, K, v, ev);
      }
    }
    if constexpr (STATS) {
      if (I.stats) curved_stats<P, LAW, T>(s, I.stats, v, ev, caps, iters, nudged);
    }
    return;
  }
  // ---------------- D: subcell fluxes (line prefix sums) and nodal alpha-tilde
  __syncthreads();  // all reads of the subcell-face fluxes done
  {
    V vrx, vry;
#pragma unroll
    for (int q = 0; q < NC; ++q) { vrx.v[q] = rx[q]; vry.v[q] = ry[q]; }
    s.Gx[t] = vrx;
    s.Gy[t] = vry;
  }
  __syncthreads();
  T xp[NC], xm[NC], yp[NC], ym[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) { xm[q] = T(0); ym[q] = T(0); }
#pragma unroll
  for (int c = 0; c < P; ++c) {
    if (c < b) {
      const V r = s.Gx[lx + c];
#pragma unroll
      for (int q = 0; q < NC; ++q) xm[q] += r.v[q];
    }
    if (c < a) {
      const V r = s.Gy[ly + c * n];
#pragma unroll
      for (int q = 0; q < NC; ++q) ym[q] += r.v[q];
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    xp[q] = (b == P) ? T(0) : xm[q] + rx[q];
    yp[q] = (a == P) ? T(0) : ym[q] + ry[q];
  }
  T at = T(1);
  int iters = 0, caps = 0;
  if (act && move) {
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
  s.alpha[t] = at;
  if (I.dbg_lo && act) {
    I.dbg_lo[g] = (double)lo;
    I.dbg_hi[g] = (double)hi;
    I.dbg_K[g] = (double)K;
    I.dbg_alpha[g] = (double)at;
  }
  T u0[NC];
  if (act && I.c0 != T(0)) {
#pragma unroll
    for (int q = 0; q < NC; ++q) u0[q] = I.u0[q * N + g];
  }
  __syncthreads();
  // ---------------- E: face coefficients and limited update
  T v = T(0), ev = T(0);
  int nudged = 0;
  if (act) {
    const T axp = (b < P) ? tmin(at, s.alpha[t + 1]) : T(0);
    const T axm = (b > 0) ? tmin(at, s.alpha[t - 1]) : T(0);
    const T ayp = (a < P) ? tmin(at, s.alpha[t + n]) : T(0);
    const T aym = (a > 0) ? tmin(at, s.alpha[t - n]) : T(0);
    T fe[NC];
    T acc[NC];
    v_scale<NC>(acc, axp, xp);
    v_fma<NC>(acc, -axm, xm, acc);
    v_fma<NC>(acc, ayp, yp, acc);
    v_fma<NC>(acc, -aym, ym, acc);
    v_fma<NC>(fe, dtm, acc, uL);
    if constexpr (sizeof(T) == 4) {
      if (!(fe[0] >= lo && fe[0] <= hi))  // rare: the rounding scale only where it is needed
        nudged = accept_rounded(fe[0], lo, hi, curved_stencil_scale<P>(s, t, a, b, u[0], FX.um, FY.um) +
                                                   fabs(uL[0]) + tmax(fabs(lo), fabs(hi)) +
                                                   dtm * (fabs(axp * xp[0]) + fabs(axm * xm[0]) + fabs(ayp * yp[0]) +
                                                          fabs(aym * ym[0])));
    }
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
    if constexpr (STATS) {
      if (I.stats && move) curved_violations<P, LAW, T>(s, I, lp, e, t, a, b, fe, lo, hi, K, v, ev);
    }
  }
  if constexpr (STATS) {
    if (I.stats) curved_stats<P, LAW, T>(s, I.stats, v, ev, caps, iters, nudged);
  }
}

template <int P, class LAW, typename T, bool ELW = false, bool STATS = false>
__global__ void __launch_bounds__(CurvedGeom<P>::THREADS, CurvedMinBlocks<T>::value) k_stage_curved(const StageLaunch<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<CurvedSmem<P, LAW, T>*>(smem_raw);
  curved_stage_body<P, LAW, T, ELW, STATS>(s, A.inst, A.tab, A.lp, A.si, A.limiter, blockIdx.x);
}

// Batched stage on curved meshes: CTA blockIdx.x runs task (instance, element block) of the task
// table; all tasks of one launch share P, law and precision.
template <int P, class LAW, typename T, bool ELW = false, bool STATS = false>
__global__ void __launch_bounds__(CurvedGeom<P>::THREADS, CurvedMinBlocks<T>::value) k_stage_curved_batch(const BatchLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<CurvedSmem<P, LAW, T>*>(smem_raw);
  __shared__ Instance<T> sI;
  const int2 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  curved_stage_body<P, LAW, T, ELW, STATS>(s, sI, B.tab, B.lp, B.si, B.limiter, task.y);
}

// CFL bound of Eq. cfl-low per node on a curved mesh, m_i / (2 sum_{j != i} d_ij): subcell faces
// d = w Lambda / 2, element faces d = w lambda |n| / 2; min-reduced into *out_bits.
template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_dt_body(CurvedSmem<P, LAW, T>& s, const Instance<T>& I, const Tables<T>& tab,
                                               const LawParamsT<T>& lp, long long eb, unsigned long long* out_bits) {
  using Gm = CurvedGeom<P>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const int t = threadIdx.x, le = t / NN, i = t - le * NN, a = i / n, b = i - a * n;
  const long long e = eb * Gm::EPB + le;
  const bool act = e < (long long)I.nx * I.ny;
  T u[NC];
  typename LAW::Aux ax;
  CurvedFace<P, LAW, T> FX{}, FY{};
  bool onx, ony;
  curved_load<P, LAW>(s, I, lp, e, act, t, a, b, u, ax, FX, FY, onx, ony);
  const T big = T(FLT_MAX);
  T val = big;
  if (act) {
    const T wa = tab.w[a], wb = tab.w[b];
    const T half = T(0.5);
    T sumd = T(0);
    sumd += (b > 0) ? half * wa * s.lam[t - 1][0] : half * wa * FX.ln;
    sumd += (b < P) ? half * wa * s.lam[t][0] : half * wa * FX.ln;
    sumd += (a > 0) ? half * wb * s.lam[t - n][1] : half * wb * FY.ln;
    sumd += (a < P) ? half * wb * s.lam[t][1] : half * wb * FY.ln;
    if (sumd > T(0)) val = fdiv(I.geo[GEO_MASS * I.N + e * NN + i], T(2) * sumd);
  }
  // block minimum: the block size need not be a multiple of 32 (EPB whole elements), so the
  // values go through shared memory and only the first, always complete, warp shuffles
  __shared__ T red[Gm::THREADS];
  red[t] = val;
  __syncthreads();
  if (t < 32) {
    val = big;
    for (int j = t; j < Gm::THREADS; j += 32) val = tmin(val, red[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val = tmin(val, __shfl_xor_sync(0xffffffffu, val, o));
    if (t == 0 && val < big) atomicMin(out_bits, (unsigned long long)__double_as_longlong((double)val));
  }
}

template <int P, class LAW, typename T>
__global__ void __launch_bounds__(CurvedGeom<P>::THREADS, CurvedMinBlocks<T>::value) k_dt_curved(const StageLaunch<T> A, unsigned long long* out_bits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<CurvedSmem<P, LAW, T>*>(smem_raw);
  curved_dt_body<P, LAW, T>(s, A.inst, A.tab, A.lp, blockIdx.x, out_bits);
}

// Batched time step on curved meshes: task (instance, element block), into the instance's accumulator.
template <int P, class LAW, typename T>
__global__ void __launch_bounds__(CurvedGeom<P>::THREADS, CurvedMinBlocks<T>::value) k_dt_curved_batch(const BatchLaunch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<CurvedSmem<P, LAW, T>*>(smem_raw);
  __shared__ Instance<T> sI;
  const int2 task = B.tasks[blockIdx.x];
  load_instance(sI, B.insts + task.x);
  curved_dt_body<P, LAW, T>(s, sI, B.tab, B.lp, task.y, B.bits + task.x);
}

template <int P, class LAW, typename T>
cudaError_t launch_curved(const StageLaunch<T>& a, unsigned long long* dt_bits, cudaStream_t s) {
  if constexpr (HasPosition<LAW>::value) {
    return cudaErrorInvalidValue;  // position-dependent laws are defined on Cartesian meshes only
  } else {
    using Gm = CurvedGeom<P>;
    constexpr size_t smem = sizeof(CurvedSmem<P, LAW, T>);
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t err = cudaFuncSetAttribute(k_stage_curved<P, LAW, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      err = cudaFuncSetAttribute(k_stage_curved<P, LAW, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      err = cudaFuncSetAttribute(k_stage_curved<P, LAW, T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      err = cudaFuncSetAttribute(k_stage_curved<P, LAW, T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      err = cudaFuncSetAttribute(k_dt_curved<P, LAW, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      attr_set = true;
    }
    const long long Ne = (long long)a.inst.nx * a.inst.ny;
    const long long blocks = (Ne + Gm::EPB - 1) / Gm::EPB;
    if (blocks <= 0) return cudaSuccess;
    const bool elw = a.limiter == SIDP_LIMITER_ELEMENTWISE, stats = a.inst.stats && a.limiter >= 2;
    if (dt_bits) k_dt_curved<P, LAW, T><<<(unsigned)blocks, Gm::THREADS, smem, s>>>(a, dt_bits);
    else if (elw && stats) k_stage_curved<P, LAW, T, true, true><<<(unsigned)blocks, Gm::THREADS, smem, s>>>(a);
    else if (elw) k_stage_curved<P, LAW, T, true><<<(unsigned)blocks, Gm::THREADS, smem, s>>>(a);
    else if (stats) k_stage_curved<P, LAW, T, false, true><<<(unsigned)blocks, Gm::THREADS, smem, s>>>(a);
    else k_stage_curved<P, LAW, T><<<(unsigned)blocks, Gm::THREADS, smem, s>>>(a);
    return cudaGetLastError();
  }
}

// Batched launches on curved meshes: the tasks are (instance, element block of EPB elements).
template <int P, class LAW, typename T>
cudaError_t launch_curved_batch(const BatchLaunch<T>& B, bool dt, cudaStream_t s) {
  if constexpr (HasPosition<LAW>::value) {
    return cudaErrorInvalidValue;  // position-dependent laws are defined on Cartesian meshes only
  } else {
    using Gm = CurvedGeom<P>;
    constexpr size_t smem = sizeof(CurvedSmem<P, LAW, T>);
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t err = cudaSuccess;
      auto set = [&](const void* f) {
        if (err == cudaSuccess) err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      };
      set((const void*)k_stage_curved_batch<P, LAW, T>);
      set((const void*)k_stage_curved_batch<P, LAW, T, true>);
      set((const void*)k_stage_curved_batch<P, LAW, T, false, true>);
      set((const void*)k_stage_curved_batch<P, LAW, T, true, true>);
      set((const void*)k_dt_curved_batch<P, LAW, T>);
      if (err != cudaSuccess) return err;
      attr_set = true;
    }
    if (B.ntasks <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)B.ntasks;
    const bool elw = B.limiter == SIDP_LIMITER_ELEMENTWISE, stats = B.stats && B.limiter >= 2;
    if (dt) k_dt_curved_batch<P, LAW, T><<<grid, Gm::THREADS, smem, s>>>(B);
    else if (elw && stats) k_stage_curved_batch<P, LAW, T, true, true><<<grid, Gm::THREADS, smem, s>>>(B);
    else if (elw) k_stage_curved_batch<P, LAW, T, true><<<grid, Gm::THREADS, smem, s>>>(B);
    else if (stats) k_stage_curved_batch<P, LAW, T, false, true><<<grid, Gm::THREADS, smem, s>>>(B);
    else k_stage_curved_batch<P, LAW, T><<<grid, Gm::THREADS, smem, s>>>(B);
    return cudaGetLastError();
  }
}

}  // namespace sidp
