// Line-parallel stage kernel on curved (mapped) quadrilateral meshes: the curved-mesh update of
// `k_stage_curved` (Sec. 2.3 metric terms, the conservative metric correction of Sec. 3.1, the
// low-order operator Eq. dg-lo-modified, subcell limiting of Sec. 4.1.3 and 4.3, SSP-RK3 of Sec. 5)
// with one thread per element line, as `k_stage_lines` does on Cartesian meshes.
//
// A CTA owns E whole elements (no tile halo: every element face is evaluated inside the element
// from the node's own state and the neighbour's trace, read from global memory, L2-resident).
// Thread j of element K is the thread of row j and of column j of K:
//   A  the row's state, contravariant rows r1, corrected rows q1 and masses by vector loads; the
//      row's per-node quantities and sigma into shared memory;
//   B  column role: the element-face items of the column (normals and neighbour traces, loaded at
//      the start of the role: loaded in phase A they stayed live across the barrier and spilled),
//      the column's nodes from shared memory, its rows r2 / q2 from global memory;
//      y subcell faces (Lambda over both nodes' corrected rows, two bar states), the two element
//      faces, the contraction of r2 . F with D_1D, r^H_y, r^L_y, bounds and prefix sums -> shared
//      memory for the row threads;
//   C  row role: the same along x;
//   D, E  as in `k_stage_lines` (u^L, bounds, Zalesak, the entropy line search, the limited
//      update with the masses m_i = w_a w_b G_i of the mesh).
// Both elements of a face evaluate it from the same operands in the same order (the -xi/-eta side
// as the left state), so the update is conservative up to the rounding of the final sums.
#pragma once
#include "sidp_curved.cuh"
#include "sidp_lines.cuh"

namespace sidp {

template <int P>
struct CurvedLineGeom {
  static constexpr int n = P + 1, NN = n * n;
  static constexpr int E = (128 / n) > 0 ? 128 / n : 1;  // elements per CTA (32 at p = 3)
  static constexpr int NL = E * n;
  static constexpr int THREADS = ((NL + 31) / 32) * 32;
  static constexpr bool SWZ = (n == 4);  // rotated rows, as in LineGeom
  static constexpr int SE = SWZ ? NN : NN + (NN == 4 ? 2 : NN == 64 ? 8 : 0);
  static constexpr int NTP = ((E * SE + 3) / 4) * 4;
  __device__ __forceinline__ static int rs(int le, int a) {
    if constexpr (SWZ) return le * SE + n * ((a + (le >> 1)) & 3);
    else return le * SE + n * a;
  }
};

template <int P, class LAW, typename T>
struct CurvedLineSmem {
  using G = CurvedLineGeom<P>;
  static constexpr int NC = LAW::NC, NA = AuxWords<LAW, T>::value;
  T u[NC][G::NTP];
  T aux[NA > 0 ? NA : 1][G::NTP];
  T sig[LAW::kEntropy ? G::NTP : 4];
  T rly[NC][G::NTP];
  T sy[NC][G::NTP];
  T lo[G::NTP];
  T hi[G::NTP];
  T K[LAW::kEntropy ? G::NTP : 4];
  T alpha[G::NTP];
  T umS[G::NL + 4], umN[G::NL + 4];  // |u| of the neighbour traces across the S and N faces, per column
};

// An element face of a line as seen from its node: the face normal and the neighbour's trace (or
// ext = false at an outflow or slip-wall side, where the ghost is built from the own trace).
template <class LAW, typename T>
struct CurvedItem {
  T un[LAW::NC];
  T nvx, nvy;
  bool ext;
};

template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_item_load(const Instance<T>& I, long long e, int a, int b, int side,
                                                 CurvedItem<LAW, T>& it) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  const long long N = I.N, gi = e * NN + a * n + b;
  const int dir = side >> 1;
  it.nvx = I.geo[(dir == 0 ? GEO_NXX : GEO_NYX) * N + gi];
  it.nvy = I.geo[(dir == 0 ? GEO_NXY : GEO_NYY) * N + gi];
  const long long gn = curved_nbr<P>(I.bc, I.nx, I.ny, e, a, b, side);
  it.ext = gn >= 0;
#pragma unroll
  for (int q = 0; q < NC; ++q) it.un[q] = it.ext ? I.uin[q * N + gn] : T(0);
}

// The element face of item `it` (side 0 W, 1 E, 2 S, 3 N) from the node's own state uo, ao and
// fluxes fox, foy: the same ghost, operand order and arithmetic as the node layout's face_eval.
template <class LAW, typename T>
__device__ __forceinline__ void curved_face_line(const Instance<T>& I, const LawParamsT<T>& lp, int side,
                                                 const CurvedItem<LAW, T>& it, const T* uo,
                                                 const typename LAW::Aux& ao, const T* fox, const T* foy,
                                                 CurvedFace<1, LAW, T>& F) {
  constexpr int NC = LAW::NC;
  using Aux = typename LAW::Aux;
  T un[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) un[q] = it.ext ? it.un[q] : uo[q];
  if constexpr (NC == 4) {
    if (!it.ext && I.bc[side] == SIDP_BC_SLIP_WALL) {
      const T inn = frcp(psqrt(it.nvx * it.nvx + it.nvy * it.nvy));
      const T nx = it.nvx * inn, ny = it.nvy * inn;
      const T mn = uo[1] * nx + uo[2] * ny;
      un[1] = uo[1] - T(2) * mn * nx;
      un[2] = uo[2] - T(2) * mn * ny;
    }
  }
  Aux an;
  LAW::aux(un, an, lp);
  const bool low = (side & 1) == 0;  // the neighbour is the left state
  T uL[NC], uR[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    uL[q] = low ? un[q] : uo[q];
    uR[q] = low ? uo[q] : un[q];
  }
  const Aux aL = low ? an : ao, aR = low ? ao : an;
  T fnx[NC], fny[NC];
  LAW::flux(un, an, 0, fnx, lp);
  LAW::flux(un, an, 1, fny, lp);
  T fLx[NC], fLy[NC], fRx[NC], fRy[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    fLx[q] = low ? fnx[q] : fox[q];
    fLy[q] = low ? fny[q] : foy[q];
    fRx[q] = low ? fox[q] : fnx[q];
    fRy[q] = low ? foy[q] : fny[q];
  }
  const T nvx = it.nvx, nvy = it.nvy;
  const T nn = psqrt(nvx * nvx + nvy * nvy);
  const T lam = LAW::lam_n(uL, aL, uR, aR, fdiv(nvx, nn), fdiv(nvy, nn), lp);
  F.ln = lam * nn;
  {
    T sx[NC], sy[NC], du[NC];
    v_add<NC>(sx, fLx, fRx);
    v_add<NC>(sy, fLy, fRy);
    v_scale<NC>(sx, nvx, sx);
    v_fma<NC>(sx, nvy, sy, sx);
    v_scale<NC>(sx, T(0.5), sx);
    v_sub<NC>(du, uR, uL);
    v_fma<NC>(F.Fh, T(-0.5) * F.ln, du, sx);
    v_scale<NC>(F.Fn, nvx, fox);
    v_fma<NC>(F.Fn, nvy, foy, F.Fn);
  }
  const T dF = (fRx[0] - fLx[0]) * nvx + (fRy[0] - fLy[0]) * nvy;
  F.bar = T(0.5) * (uL[0] + uR[0]) - ((F.ln > T(0)) ? fdiv(dF, T(2) * F.ln) : T(0));
  if constexpr (LAW::kEntropy) F.sig = LAW::sigma(un, an, lp);
  else F.sig = T(0);
  F.um = fabs(un[0]);
}

// One direction of one element line on a curved mesh: the line's nodes nd (state, per-node
// quantities, sigma) with their fluxes fx, fy and metric rows r (high order) and q (corrected), the
// two element faces Fl (left/lower) and Fr (right/upper); outputs per node r^L (rl), the bounds and
// K from the node and its two faces on this line, and the prefix sums S at the P subcell faces.
// w: the quadrature weight of the line (w_a of a row, w_b of a column).
template <int P, class LAW, typename T>
__device__ __forceinline__ void curved_line_residuals(const Tables<T>& tab, const LawParamsT<T>& lp,
                                                      const LNode<LAW, T>* nd, const T (*fx)[LAW::NC],
                                                      const T (*fy)[LAW::NC], const T (*r)[2], const T (*qr)[2],
                                                      const CurvedFace<1, LAW, T>& Fl, const CurvedFace<1, LAW, T>& Fr,
                                                      T w, T (*rl)[LAW::NC], T* lo, T* hi, T* K, T (*S)[LAW::NC]) {
  constexpr int n = P + 1, NC = LAW::NC;
  T f[n][NC], g[n][NC];
#pragma unroll
  for (int c = 0; c < n; ++c) {  // contravariant fluxes: (G J^-1 row) . F and (corrected row) . F
    v_scale<NC>(f[c], r[c][1], fy[c]);
    v_fma<NC>(f[c], r[c][0], fx[c], f[c]);
    v_scale<NC>(g[c], qr[c][1], fy[c]);
    v_fma<NC>(g[c], qr[c][0], fx[c], g[c]);
  }
  T sx[n][NC];
#pragma unroll
  for (int b = 0; b < n; ++b) {
#pragma unroll
    for (int q = 0; q < NC; ++q) sx[b][q] = T(0);
#pragma unroll
    for (int c = 0; c < n; ++c) v_fma<NC>(sx[b], tab.D[b * n + c], f[c], sx[b]);
  }
  // subcell faces c - 1/2 (c = 1..P): the flux G and the bar states of the lower and upper node
  T Gf[n][NC], barLo[n], barHi[n];
#pragma unroll
  for (int c = 1; c < n; ++c) {
    const LNode<LAW, T>& L = nd[c - 1];
    const LNode<LAW, T>& R = nd[c];
    const T qLx = qr[c - 1][0], qLy = qr[c - 1][1], qRx = qr[c][0], qRy = qr[c][1];
    const T nL = psqrt(qLx * qLx + qLy * qLy), nR = psqrt(qRx * qRx + qRy * qRy);
    const T lR = LAW::lam_n(L.u, L.ax, R.u, R.ax, fdiv(qRx, nR), fdiv(qRy, nR), lp) * nR;
    const T lL = LAW::lam_n(L.u, L.ax, R.u, R.ax, fdiv(qLx, nL), fdiv(qLy, nL), lp) * nL;
    const T Lam = tmax(lR, lL);
    T gs[NC], du[NC];
    v_add<NC>(gs, g[c - 1], g[c]);
    v_sub<NC>(du, R.u, L.u);
    v_scale<NC>(gs, T(0.5), gs);
    v_fma<NC>(Gf[c], T(-0.5) * Lam, du, gs);
    const T dFx = fx[c][0] - fx[c - 1][0], dFy = fy[c][0] - fy[c - 1][0];
    const T mid = T(0.5) * (L.u[0] + R.u[0]);
    const T inv2 = (Lam > T(0)) ? fdiv(T(1), T(2) * Lam) : T(0);
    barLo[c] = mid - (qRx * dFx + qRy * dFy) * inv2;  // for the lower (left) node
    barHi[c] = mid - (qLx * dFx + qLy * dFy) * inv2;  // for the upper (right) node
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {  // element-face terms of the high-order residual
    sx[0][q] += Fl.Fn[q] - Fl.Fh[q];
    sx[P][q] += Fr.Fh[q] - Fr.Fn[q];
  }
  T acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = T(0);
#pragma unroll
  for (int b = 0; b < n; ++b) {
    T rH[NC], tq[NC], rr[NC];
    v_scale<NC>(rH, -w, sx[b]);
    const T* gr = (b < P) ? Gf[b < P ? b + 1 : b] : Fr.Fh;
    const T* gl = (b > 0) ? Gf[b > 0 ? b : 1] : Fl.Fh;
    v_sub<NC>(tq, gr, gl);
    v_scale<NC>(rl[b], -w, tq);
    v_sub<NC>(rr, rH, rl[b]);
    const T bl = (b > 0) ? barHi[b > 0 ? b : 1] : Fl.bar, br = (b < P) ? barLo[b < P ? b + 1 : b] : Fr.bar;
    lo[b] = tmin(nd[b].u[0], tmin(bl, br));
    hi[b] = tmax(nd[b].u[0], tmax(bl, br));
    const T sl = (b > 0) ? nd[b > 0 ? b - 1 : 0].s : Fl.sig, sr = (b < P) ? nd[b < P ? b + 1 : b].s : Fr.sig;
    K[b] = tmin(nd[b].s, tmin(sl, sr));
    if (b < P) {
      v_add<NC>(acc, acc, rr);
#pragma unroll
      for (int q = 0; q < NC; ++q) S[b][q] = acc[q];
    }
  }
}

// Statistics of row node (j, b) of element e on a curved mesh: the entropy-bound violation as in
// the node layout (K_i from the stage input of the node and its four neighbours, accurate sigma in
// float64; across an element face the neighbour's trace, an outflow or wall ghost keeping the
// node's own sigma).
template <int P, class LAW, typename T, class S>
__device__ __forceinline__ double curved_line_entropy_violation64(const S& s, const Instance<T>& I,
                                                                  const LawParamsT<T>& lp, long long e, int le,
                                                                  int j, int b, const T* fe) {
  using G = CurvedLineGeom<P>;
  constexpr int n = P + 1, NC = LAW::NC;
  auto sig = [&](const T* u) { return (double)LAW::rhoe(u) * (double)powf(u[0], -lp.gamma); };
  auto sig_slot = [&](int slot) {
    T uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = s.u[q][slot];
    return sig(uu);
  };
  const int me = G::rs(le, j) + b;
  double K = sig_slot(me);
  if (b > 0) K = fmin(K, sig_slot(me - 1));
  if (b < P) K = fmin(K, sig_slot(me + 1));
  if (j > 0) K = fmin(K, sig_slot(G::rs(le, j - 1) + b));
  if (j < P) K = fmin(K, sig_slot(G::rs(le, j + 1) + b));
  const int sides[2] = {b == 0 ? 0 : (b == P ? 1 : -1), j == 0 ? 2 : (j == P ? 3 : -1)};
  for (int k = 0; k < 2; ++k) {
    if (sides[k] < 0) continue;
    const long long gn = curved_nbr<P>(I.bc, I.nx, I.ny, e, j, b, sides[k]);
    if (gn < 0) continue;
    T un[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) un[q] = I.uin[q * I.N + gn];
    K = fmin(K, sig(un));
  }
  if (!((double)fe[0] > 0.0)) return 1.0;
  return fmax(0.0, 1.0 - sig(fe) / K);
}

template <int P, class LAW, typename T, bool STATS>
__device__ __forceinline__ void curved_lines_body(CurvedLineSmem<P, LAW, T>& s, const Instance<T>& I,
                                                  const Tables<T>& tab, const LawParamsT<T>& lp, long long eb) {
  using G = CurvedLineGeom<P>;
  using Nd = LNode<LAW, T>;
  using Face = CurvedFace<1, LAW, T>;
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC, NA = AuxWords<LAW, T>::value;
  const int t = threadIdx.x;
  const bool live = (G::NL == G::THREADS) || (t < G::NL);
  const int le = live ? t / n : 0, j = live ? t - le * n : 0;
  const long long e = eb * G::E + le;
  const bool act = live && e < (long long)I.nx * I.ny;
  const long long N = I.N;
  const long long ge = act ? e : 0;                 // the element whose data a thread reads
  const long long grow = ge * NN + j * n;           // global index of node (j, 0)
  const int srow = G::rs(le, j);
  const T wj = pick<n>(tab.w, j);
  const T dt = *I.dtT;
  const bool move = (dt > T(0)) && (dt < T(FLT_MAX));
  const T* geo = I.geo;

  // ---------------- A: the row
  T ur[NC][n], r1[2][n], q1[2][n], mr[n];
#pragma unroll
  for (int q = 0; q < NC; ++q) ld_line<n>(I.uin + q * N + grow, ur[q]);
  ld_line<n>(geo + GEO_R1X * N + grow, r1[0]);
  ld_line<n>(geo + GEO_R1Y * N + grow, r1[1]);
  ld_line<n>(geo + GEO_Q1X * N + grow, q1[0]);
  ld_line<n>(geo + GEO_Q1Y * N + grow, q1[1]);
  ld_line<n>(geo + GEO_MASS * N + grow, mr);
  if (live) {
    T sg[n];
    typename LAW::Aux ax[n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T uu[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) uu[q] = ur[q][b];
      LAW::aux(uu, ax[b], lp);
      sg[b] = LAW::kEntropy ? LAW::sigma(uu, ax[b], lp) : T(0);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) st_line<n>(&s.u[q][srow], ur[q]);
    if constexpr (NA > 0) {
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        T v[n];
#pragma unroll
        for (int b = 0; b < n; ++b) v[b] = reinterpret_cast<const T*>(&ax[b])[k];
        st_line<n>(&s.aux[k][srow], v);
      }
    }
    if constexpr (LAW::kEntropy) st_line<n>(&s.sig[srow], sg);
  }
  __syncthreads();

  // ---------------- B: column role (column j of element le)
  if (live) {
    CurvedItem<LAW, T> itS, itN;
    curved_item_load<P, LAW>(I, ge, 0, j, 2, itS);
    curved_item_load<P, LAW>(I, ge, P, j, 3, itN);
    Nd nd[n];
    T fx[n][NC], fy[n][NC], r2[n][2], q2[n][2];
#pragma unroll
    for (int a = 0; a < n; ++a) {
      const int sl = G::rs(le, a) + j;
      ld_node<LAW, T>(s, sl, nd[a]);
      LAW::flux(nd[a].u, nd[a].ax, 0, fx[a], lp);
      LAW::flux(nd[a].u, nd[a].ax, 1, fy[a], lp);
      const long long gi = ge * NN + a * n + j;
      r2[a][0] = geo[GEO_R2X * N + gi];
      r2[a][1] = geo[GEO_R2Y * N + gi];
      q2[a][0] = geo[GEO_Q2X * N + gi];
      q2[a][1] = geo[GEO_Q2Y * N + gi];
    }
    Face FS, FN;
    curved_face_line<LAW, T>(I, lp, 2, itS, nd[0].u, nd[0].ax, fx[0], fy[0], FS);
    curved_face_line<LAW, T>(I, lp, 3, itN, nd[P].u, nd[P].ax, fx[P], fy[P], FN);
    T rl[n][NC], lo[n], hi[n], K[n], S[n][NC];
    curved_line_residuals<P, LAW, T>(tab, lp, nd, fx, fy, r2, q2, FS, FN, wj, rl, lo, hi, K, S);
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
    s.umS[le * n + j] = FS.um;
    s.umN[le * n + j] = FN.um;
  }

  // ---------------- C: row role (row j of element le)
  T rlx[n][NC], lox[n], hix[n], Kx[n], Sx[n][NC];
  Face FW, FE;
  if (live) {
    CurvedItem<LAW, T> itW, itE;
    curved_item_load<P, LAW>(I, ge, j, 0, 0, itW);
    curved_item_load<P, LAW>(I, ge, j, P, 1, itE);
    Nd nd[n];
    T fx[n][NC], fy[n][NC], rr[n][2], qq[n][2];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      ld_node<LAW, T>(s, srow + b, nd[b]);
      LAW::flux(nd[b].u, nd[b].ax, 0, fx[b], lp);
      LAW::flux(nd[b].u, nd[b].ax, 1, fy[b], lp);
      rr[b][0] = r1[0][b];
      rr[b][1] = r1[1][b];
      qq[b][0] = q1[0][b];
      qq[b][1] = q1[1][b];
    }
    curved_face_line<LAW, T>(I, lp, 0, itW, nd[0].u, nd[0].ax, fx[0], fy[0], FW);
    curved_face_line<LAW, T>(I, lp, 1, itE, nd[P].u, nd[P].ax, fx[P], fy[P], FE);
    curved_line_residuals<P, LAW, T>(tab, lp, nd, fx, fy, rr, qq, FW, FE, wj, rlx, lox, hix, Kx, Sx);
  }
  __syncthreads();

  // ---------------- D: per node of the row, u^L, bounds and alpha-tilde (as in k_stage_lines, with
  // the mesh's masses m_i)
  T uL[n][NC], at[n], dtm[n], lob[n], hib[n], kb[n];
  T yp[n][NC], ym[n][NC];
  int iters = 0, caps = 0;
  if (live) {
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
    unsigned slow = 0;
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const T m = mr[b];
      dtm[b] = move ? fdiv(dt, m) : T(0);
      T tq[NC], uu[NC], rr[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) { uu[q] = ur[q][b]; rr[q] = rly[q][b]; }
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
      if (act && move) {
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
  T u0[NC][n];
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
        if (act && !(fe[0] >= lob[b] && fe[0] <= hib[b])) {  // rare: the rounding scale only where it is needed
          const int me = srow + b;
          const T sl = (b > 0) ? fabs(s.u[0][me - 1]) : FW.um, sr = (b < P) ? fabs(s.u[0][me + 1]) : FE.um;
          const T sd = (j > 0) ? fabs(s.u[0][G::rs(le, j > 0 ? j - 1 : 0) + b]) : s.umS[le * n + b];
          const T su = (j < P) ? fabs(s.u[0][G::rs(le, j < P ? j + 1 : 0) + b]) : s.umN[le * n + b];
          const T scl = fabs(ur[0][b]) + T(2) * tmax(tmax(sl, sr), tmax(sd, su));
          const T mag = scl + fabs(uL[b][0]) + tmax(fabs(lob[b]), fabs(hib[b])) +
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
              ev = T(curved_line_entropy_violation64<P, LAW, T>(s, I, lp, e, le, j, b, fe));
            } else {
              ev = tmax(T(0), T(1) - LAW::sigma_of(fe, lp) / kb[b]);
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
      } else {
        T r1v[NC], uu[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) uu[q] = u0[q][b];
        v_scale<NC>(r1v, I.c1, fe);
        v_fma<NC>(r1v, I.c0, uu, r1v);
#pragma unroll
        for (int q = 0; q < NC; ++q) res[q][b] = r1v[q];
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

template <int P, class LAW, typename T>
struct CurvedLineBounds {
  using G = CurvedLineGeom<P>;
  static constexpr int SMEM_CTAS = (int)((227u * 1024u) / (sizeof(CurvedLineSmem<P, LAW, T>) + 1024u));
  static constexpr int REG_CTAS = 65536 / (G::THREADS * 128);
  static constexpr int M = SMEM_CTAS < REG_CTAS ? SMEM_CTAS : REG_CTAS;
  static constexpr int MINB = M < 1 ? 1 : M;
};

template <int P, class LAW, typename T, bool STATS>
__global__ void __launch_bounds__(CurvedLineGeom<P>::THREADS, (CurvedLineBounds<P, LAW, T>::MINB))
k_stage_curved_lines(const StageLaunch<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& s = *reinterpret_cast<CurvedLineSmem<P, LAW, T>*>(smem_raw);
  curved_lines_body<P, LAW, T, STATS>(s, A.inst, A.tab, A.lp, blockIdx.x);
}

// The curved line kernel of one law: Euler only (the other laws run the node layout).
template <int P, class LAW, typename T>
struct CurvedLines {
  static cudaError_t stage(const StageLaunch<T>&, bool, cudaStream_t) { return cudaErrorInvalidValue; }
};

template <int P, typename T>
struct CurvedLines<P, LawEuler<T>, T> {
  static cudaError_t stage(const StageLaunch<T>& a, bool stats, cudaStream_t s) {
    using G = CurvedLineGeom<P>;
    using LAW = LawEuler<T>;
    constexpr size_t smem = sizeof(CurvedLineSmem<P, LAW, T>);
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t err = cudaFuncSetAttribute(k_stage_curved_lines<P, LAW, T, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_stage_curved_lines<P, LAW, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
      if (err != cudaSuccess) return err;
      attr_set = true;
    }
    const long long Ne = (long long)a.inst.nx * a.inst.ny;
    const long long blocks = (Ne + G::E - 1) / G::E;
    if (blocks <= 0) return cudaSuccess;
    if (stats) k_stage_curved_lines<P, LAW, T, true><<<(unsigned)blocks, G::THREADS, smem, s>>>(a);
    else k_stage_curved_lines<P, LAW, T, false><<<(unsigned)blocks, G::THREADS, smem, s>>>(a);
    return cudaGetLastError();
  }
};

}  // namespace sidp
