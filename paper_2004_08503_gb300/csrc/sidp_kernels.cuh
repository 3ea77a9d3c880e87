// Fused stage kernel and CFL time-step kernel, templated on degree P, law and precision T.
//
// One CTA owns EPB elements; one thread owns one node (a, b) of one element.  A stage is
// element-local once the 4(p+1) face-neighbour nodes are known, so the whole forward-Euler
// update (Sec. 4, Eq. subcell-fct / convex-fct) plus the SSP-RK3 combination (Sec. 5) runs in
// one kernel with three CTA barriers:
//   A  load u (coalesced, element-major SoA) and the one face-neighbour node this thread
//      touches in x and in y; node aux (velocity, pressure, sound speed), fluxes F_x, F_y and
//      the entropy function sigma into shared memory
//   B  subcell faces: thread b evaluates the x face to its left (q = b; q = 0 is the element
//      face, with the neighbour's trace) and thread b = p also the right element face (q = n).
//      Each face stores its flux -- the Lax-Friedrichs flux Eq. lax-friedrichs on element faces,
//      the Rusanov flux of the sparsified operator on interior subcell faces (Eq. dg-idp with
//      D-hat of Eq. didp and d_ij of Eq. dij) -- and the bar state of the limited field
//      (Eq. bar-states).  Same for y.
//   C  r^H (strong form, Eq. ho-update: line contraction with D_1D plus face corrections),
//      r^L (difference of face fluxes), u^L, local bounds (Sec. 4.1.1 / 4.3), r = r^H - r^L
//   D  subcell fluxes r-bar (prefix sums along lines, Sec. 4.1.3), nodal alpha-tilde
//      (Zalesak on field 0; Euler: entropy line search over the gamma-scaled candidates)
//   E  alpha_{m,k} = min of the two adjacent alpha-tilde; limited update; RK combination.
// Every face flux is computed once and used by both adjacent nodes, and both elements sharing
// an element face evaluate its flux with identical (left, right) arguments, so the update is
// conservative to rounding.
#pragma once
#include <cfloat>
#include "sidp_internal.h"
#include "sidp_laws.cuh"

namespace sidp {

constexpr int kRootMaxIt = 60;

template <typename T> struct Prec;
template <> struct Prec<double> { static constexpr double root_tol = 1e-13; };
template <> struct Prec<float> { static constexpr float root_tol = 2e-6f; };

// Elements per CTA: about 256 threads; the CTA is padded to whole warps.
__host__ __device__ constexpr int epb_for(int P) { return ((P + 1) * (P + 1) >= 256) ? 1 : 256 / ((P + 1) * (P + 1)); }
__host__ __device__ constexpr int stage_threads(int P) { return ((epb_for(P) * (P + 1) * (P + 1) + 31) / 32) * 32; }

template <int P, class LAW, typename T>
struct ElemSmem {
  static constexpr int n = P + 1, NN = n * n, NC = LAW::NC, NF = n * (n + 1);
  T u[NC][NN];
  T fx[NC][NN];  // F_x at the nodes, later r_x
  T fy[NC][NN];  // F_y at the nodes, later r_y
  T sig[LAW::kEntropy ? NN : 1];
  T fbx[NC][NF];  // x-face fluxes, [f][a*(n+1) + q]
  T fby[NC][NF];  // y-face fluxes, [f][b*(n+1) + q]
  T bbx[NF];      // x-face bar state of field 0
  T bby[NF];
  T alpha[NN];
  typename LAW::Aux aux[NN];
};

template <int P, class LAW, typename T>
constexpr size_t stage_smem_bytes() {
  return epb_for(P) * sizeof(ElemSmem<P, LAW, T>) + sizeof(T) * ((P + 1) * (P + 1) + (P + 1));
}

// Trace of the neighbouring element across `side` (0 W, 1 E, 2 S, 3 N) at position `pos`
// along the face.  Outflow (reading: ghost = interior trace) copies `own`.
template <int P, int NC, typename T>
__device__ __forceinline__ void neighbor_state(const Instance<T>& I, int side, long long e, int ex, int ey,
                                               int pos, const T* own, T* out) {
  constexpr int n = P + 1, NN = n * n;
  long long ne = -1;
  int nd = 0;
  int bc = I.bc[side];
  switch (side) {
    case 0: nd = pos * n + P; ne = (ex > 0) ? e - 1 : (bc == 0 ? e + (I.nx - 1) : -1); break;
    case 1: nd = pos * n; ne = (ex < I.nx - 1) ? e + 1 : (bc == 0 ? e - (I.nx - 1) : -1); break;
    case 2: nd = P * n + pos; ne = (ey > 0) ? e - I.nx : (bc == 0 ? e + (long long)(I.ny - 1) * I.nx : -1); break;
    default: nd = pos; ne = (ey < I.ny - 1) ? e + I.nx : (bc == 0 ? e - (long long)(I.ny - 1) * I.nx : -1); break;
  }
  if (ne >= 0) {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = I.uin[f * I.N + ne * NN + nd];
  } else if (bc == 2 && I.ghost[side] != nullptr) {
    const long long nside = (side < 2) ? I.ny : I.nx;
    const long long along = (side < 2) ? ey : ex;
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = I.ghost[side][(f * nside + along) * n + pos];
  } else {
#pragma unroll
    for (int f = 0; f < NC; ++f) out[f] = own[f];
  }
}

// Face between left state L and right state R along +e_k: Rusanov / LF flux and bar state of field 0.
template <class LAW, typename T>
__device__ __forceinline__ void face_eval(int k, const T* uL, const typename LAW::Aux& aL, const T* FL,
                                          const T* uR, const typename LAW::Aux& aR, const T* FR,
                                          const LawParams& lp, T* fb, T& bar0) {
  constexpr int NC = LAW::NC;
  const T lam = LAW::lam(k, uL, aL, uR, aR, lp);
#pragma unroll
  for (int f = 0; f < NC; ++f) fb[f] = T(0.5) * (FL[f] + FR[f]) - T(0.5) * lam * (uR[f] - uL[f]);
  bar0 = (lam > T(0)) ? T(0.5) * (uL[0] + uR[0]) - (FR[0] - FL[0]) / (T(2) * lam) : T(0.5) * (uL[0] + uR[0]);
}

// Euler: largest t in [0, tcap] such that every candidate u^L + t w_c (w_c = gamma_d dt/m (+-r-bar))
// has rho > 0 and psi_K >= min(0, psi_K(u^L)).  psi_K is concave, so along each candidate the
// admissible set is an interval [0, t*]; candidates are processed in turn with the running cap.
// Root search: bracket [tL feasible, tR infeasible]; chord from the feasible end (stays feasible
// by concavity) and tangent from the infeasible end (stays infeasible), each classified by an
// actual evaluation, with a bisection step whenever the bracket did not halve.  Bounded by
// kRootMaxIt iterations (then the feasible end is returned and the cap is counted).
template <class LAW, typename T>
__device__ T entropy_limit(const T* uL, T K, const T (*cand)[4], T tcap, const LawParams& lp,
                           int& iters, int& caps) {
  const T psi0 = LAW::psi(uL, K, lp);
  const T target = tmin(psi0, T(0));
  T t = tcap;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    if (!(t > T(0))) break;
    const T* w = cand[c];
    T ut[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) ut[f] = uL[f] + t * w[f];
    if (ut[0] > T(0) && LAW::psi(ut, K, lp) >= target) continue;
    T tL = T(0), fL = psi0 - target, tR = t;
    if (w[0] < T(0)) {
      const T t0 = -uL[0] / w[0];
      if (t0 < tR) tR = t0;
    }
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
        // chord root (feasible side)
        T tc = tL + fL * (tR - tL) / (fL - fR);
        if (tc > tL && tc < tR) {
          T uc[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) uc[f] = uL[f] + tc * w[f];
          const T fc = (uc[0] > T(0)) ? LAW::psi(uc, K, lp) - target : T(-1);
          if (uc[0] > T(0) && fc >= T(0)) { tL = tc; fL = fc; } else { tR = tc; }
        }
        // tangent root from tR (infeasible side)
        const T dR = LAW::psi_grad_dot(uR, K, w, lp);
        if (dR < T(0)) {
          const T tn = tR - fR / dR;
          if (tn > tL && tn < tR) {
            T un[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) un[f] = uL[f] + tn * w[f];
            const T fn = (un[0] > T(0)) ? LAW::psi(un, K, lp) - target : T(-1);
            if (un[0] > T(0) && fn >= T(0)) { tL = tn; fL = fn; } else { tR = tn; }
          }
        }
      }
      if (tR - tL > T(0.5) * width) {  // ensure at least halving
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
    t = tL;
  }
  return t;
}

template <typename T>
__device__ __forceinline__ void block_max_atomic(T v, unsigned long long* dst) {
  // v >= 0; reduce in the warp then one atomic per warp on the double bit pattern
  double d = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0 && d > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(d));
}

template <int P, class LAW, typename T>
__global__ void __launch_bounds__(stage_threads(P))
k_stage(const StageLaunch<T> A) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC, NF = n * (n + 1), EPB = epb_for(P);
  using Aux = typename LAW::Aux;
  using ES = ElemSmem<P, LAW, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ES* S = reinterpret_cast<ES*>(smem_raw);
  T* sD = reinterpret_cast<T*>(S + EPB);
  T* sw = sD + NN;

  const Instance<T>& I = A.inst;
  const LawParams& lp = A.lp;
  const int tid = threadIdx.x;
  const int le = tid / NN, node = tid - le * NN;
  const int a = node / n, b = node - a * n;
  const long long Ne = (long long)I.nx * I.ny;
  const long long e = (long long)blockIdx.x * EPB + le;
  const bool act = (le < EPB) && (e < Ne);
  const int ex = act ? (int)(e % I.nx) : 0, ey = act ? (int)(e / I.nx) : 0;
  ES& s = S[le < EPB ? le : 0];
  if (tid < NN) sD[tid] = A.tab.D[tid];
  if (tid < n) sw[tid] = A.tab.w[tid];

  const double dtd = *I.dt;
  const T dt = T(dtd);
  const bool move = (dtd > 0.0) && (dtd < DBL_MAX);
  const long long N = I.N;
  const long long g = e * NN + node;
  const T h = T(I.h);

  // ---------------- A: node state, aux, fluxes, sigma; face-neighbour traces
  T u[NC], fx[NC], fy[NC], hx[NC], hy[NC];
  Aux ax, ahx, ahy;
  T sig = T(0), Kh = T(FLT_MAX);
  if (act) {
#pragma unroll
    for (int f = 0; f < NC; ++f) u[f] = I.uin[f * N + g];
    if (b == 0) neighbor_state<P, NC>(I, 0, e, ex, ey, a, u, hx);
    else if (b == P) neighbor_state<P, NC>(I, 1, e, ex, ey, a, u, hx);
    if (a == 0) neighbor_state<P, NC>(I, 2, e, ex, ey, b, u, hy);
    else if (a == P) neighbor_state<P, NC>(I, 3, e, ex, ey, b, u, hy);
    LAW::aux(u, ax, lp);
    LAW::flux(u, ax, 0, fx, lp);
    LAW::flux(u, ax, 1, fy, lp);
#pragma unroll
    for (int f = 0; f < NC; ++f) { s.u[f][node] = u[f]; s.fx[f][node] = fx[f]; s.fy[f][node] = fy[f]; }
    s.aux[node] = ax;
    if constexpr (LAW::kEntropy) { sig = LAW::sigma(u, ax, lp); s.sig[node] = sig; }
  }
  __syncthreads();

  // ---------------- B: subcell and element faces
  if (act) {
    T fb[NC], bar, tmpu[NC], tmpF[NC], hF[NC];
    // x face q = b (left of the node)
    if (b == 0) {
      LAW::aux(hx, ahx, lp);
      LAW::flux(hx, ahx, 0, hF, lp);
      face_eval<LAW>(0, hx, ahx, hF, u, ax, fx, lp, fb, bar);
      if constexpr (LAW::kEntropy) Kh = tmin(Kh, LAW::sigma(hx, ahx, lp));
    } else {
#pragma unroll
      for (int f = 0; f < NC; ++f) { tmpu[f] = s.u[f][node - 1]; tmpF[f] = s.fx[f][node - 1]; }
      face_eval<LAW>(0, tmpu, s.aux[node - 1], tmpF, u, ax, fx, lp, fb, bar);
    }
#pragma unroll
    for (int f = 0; f < NC; ++f) s.fbx[f][a * (n + 1) + b] = fb[f];
    s.bbx[a * (n + 1) + b] = bar;
    if (b == P) {  // right element face
      LAW::aux(hx, ahx, lp);
      LAW::flux(hx, ahx, 0, hF, lp);
      face_eval<LAW>(0, u, ax, fx, hx, ahx, hF, lp, fb, bar);
#pragma unroll
      for (int f = 0; f < NC; ++f) s.fbx[f][a * (n + 1) + n] = fb[f];
      s.bbx[a * (n + 1) + n] = bar;
      if constexpr (LAW::kEntropy) Kh = tmin(Kh, LAW::sigma(hx, ahx, lp));
    }
    // y face q = a (below the node)
    if (a == 0) {
      LAW::aux(hy, ahy, lp);
      LAW::flux(hy, ahy, 1, hF, lp);
      face_eval<LAW>(1, hy, ahy, hF, u, ax, fy, lp, fb, bar);
      if constexpr (LAW::kEntropy) Kh = tmin(Kh, LAW::sigma(hy, ahy, lp));
    } else {
#pragma unroll
      for (int f = 0; f < NC; ++f) { tmpu[f] = s.u[f][node - n]; tmpF[f] = s.fy[f][node - n]; }
      face_eval<LAW>(1, tmpu, s.aux[node - n], tmpF, u, ax, fy, lp, fb, bar);
    }
#pragma unroll
    for (int f = 0; f < NC; ++f) s.fby[f][b * (n + 1) + a] = fb[f];
    s.bby[b * (n + 1) + a] = bar;
    if (a == P) {
      LAW::aux(hy, ahy, lp);
      LAW::flux(hy, ahy, 1, hF, lp);
      face_eval<LAW>(1, u, ax, fy, hy, ahy, hF, lp, fb, bar);
#pragma unroll
      for (int f = 0; f < NC; ++f) s.fby[f][b * (n + 1) + n] = fb[f];
      s.bby[b * (n + 1) + n] = bar;
      if constexpr (LAW::kEntropy) Kh = tmin(Kh, LAW::sigma(hy, ahy, lp));
    }
  }
  __syncthreads();

  // ---------------- C: residuals, low-order state, bounds
  T uL[NC], rx[NC], ry[NC], uH[NC];
  T lo = T(0), hi = T(0), K = T(0);
  const T wa = sw[a], wb = sw[b];
  const T m = h * h * wa * wb;
  const T dtm = dt / m;
  if (act) {
    const T hwa = h * wa, hwb = h * wb;
#pragma unroll
    for (int f = 0; f < NC; ++f) {
      T sx = T(0), sy = T(0);
#pragma unroll
      for (int c = 0; c < n; ++c) {
        sx += sD[b * n + c] * s.fx[f][a * n + c];
        sy += sD[a * n + c] * s.fy[f][c * n + b];
      }
      const T* fbxr = &s.fbx[f][a * (n + 1)];
      const T* fbyr = &s.fby[f][b * (n + 1)];
      if (b == 0) sx += fx[f] - fbxr[0];
      if (b == P) sx += fbxr[n] - fx[f];
      if (a == 0) sy += fy[f] - fbyr[0];
      if (a == P) sy += fbyr[n] - fy[f];
      const T rHx = -hwa * sx, rHy = -hwb * sy;
      const T rLx = -hwa * (fbxr[b + 1] - fbxr[b]);
      const T rLy = -hwb * (fbyr[a + 1] - fbyr[a]);
      uL[f] = u[f] + dtm * (rLx + rLy);
      uH[f] = u[f] + dtm * (rHx + rHy);
      rx[f] = rHx - rLx;
      ry[f] = rHy - rLy;
    }
    const T* bbr = &s.bbx[a * (n + 1)];
    const T* bcl = &s.bby[b * (n + 1)];
    lo = tmin(tmin(u[0], tmin(bbr[b], bbr[b + 1])), tmin(bcl[a], bcl[a + 1]));
    hi = tmax(tmax(u[0], tmax(bbr[b], bbr[b + 1])), tmax(bcl[a], bcl[a + 1]));
    if constexpr (LAW::kEntropy) {
      K = tmin(sig, Kh);
      if (b > 0) K = tmin(K, s.sig[node - 1]);
      if (b < P) K = tmin(K, s.sig[node + 1]);
      if (a > 0) K = tmin(K, s.sig[node - n]);
      if (a < P) K = tmin(K, s.sig[node + n]);
    }
  }
  T fe[NC];
  if (A.limiter == 2) {
    __syncthreads();  // all reads of F_x, F_y done
    if (act) {
#pragma unroll
      for (int f = 0; f < NC; ++f) { s.fx[f][node] = rx[f]; s.fy[f][node] = ry[f]; }
    }
    __syncthreads();
    // ---------------- D: subcell fluxes and nodal alpha-tilde
    T xp[NC], xm[NC], yp[NC], ym[NC];
    T at = T(1);
    int iters = 0, caps = 0;
    if (act) {
#pragma unroll
      for (int f = 0; f < NC; ++f) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < P; ++c) if (c < b) acc += s.fx[f][a * n + c];
        xm[f] = acc;
        xp[f] = (b == P) ? T(0) : acc + s.fx[f][a * n + b];
        acc = T(0);
#pragma unroll
        for (int c = 0; c < P; ++c) if (c < a) acc += s.fy[f][c * n + b];
        ym[f] = acc;
        yp[f] = (a == P) ? T(0) : acc + s.fy[f][a * n + b];
      }
      if (move) {
        // Zalesak on field 0: contributions +r-bar_{m+}, -r-bar_{m-} per direction
        const T c1 = xp[0], c2 = -xm[0], c3 = yp[0], c4 = -ym[0];
        const T Pp = tmax(c1, T(0)) + tmax(c2, T(0)) + tmax(c3, T(0)) + tmax(c4, T(0));
        const T Pm = tmin(c1, T(0)) + tmin(c2, T(0)) + tmin(c3, T(0)) + tmin(c4, T(0));
        const T mdt = m / dt;
        const T Qp = tmax(T(0), mdt * (hi - uL[0]));
        const T Qm = tmin(T(0), mdt * (lo - uL[0]));
        const T Rp = (Pp > T(0)) ? tmin(T(1), Qp / Pp) : T(1);
        const T Rm = (Pm < T(0)) ? tmin(T(1), Qm / Pm) : T(1);
        at = tmin(Rp, Rm);
        if constexpr (LAW::kEntropy) {
          const T sc = T(4) * dtm;  // gamma_d = 2d = 4
          T cand[4][4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            cand[0][f] = sc * xp[f];
            cand[1][f] = -sc * xm[f];
            cand[2][f] = sc * yp[f];
            cand[3][f] = -sc * ym[f];
          }
          at = entropy_limit<LAW>(uL, K, cand, at, lp, iters, caps);
        }
      }
      s.alpha[node] = at;
      if (I.dbg_lo) {
        I.dbg_lo[g] = (double)lo;
        I.dbg_hi[g] = (double)hi;
        I.dbg_K[g] = (double)K;
        I.dbg_alpha[g] = (double)at;
      }
    }
    __syncthreads();
    // ---------------- E: face coefficients and limited update
    if (act) {
      const T axp = (b < P) ? tmin(at, s.alpha[node + 1]) : T(0);
      const T axm = (b > 0) ? tmin(at, s.alpha[node - 1]) : T(0);
      const T ayp = (a < P) ? tmin(at, s.alpha[node + n]) : T(0);
      const T aym = (a > 0) ? tmin(at, s.alpha[node - n]) : T(0);
#pragma unroll
      for (int f = 0; f < NC; ++f) fe[f] = uL[f] + dtm * (axp * xp[f] - axm * xm[f] + ayp * yp[f] - aym * ym[f]);
    }
    if (I.stats) {
      T v = T(0), ev = T(0);
      if (act && move) {
        const T scale = tmax(fabs(lo), fabs(hi));
        v = tmax(lo - fe[0], fe[0] - hi);
        v = (v > T(0)) ? v / (scale > T(0) ? scale : T(1)) : T(0);
        if constexpr (LAW::kEntropy) {
          const T sg = LAW::sigma_of(fe, lp);
          ev = tmax(T(0), T(1) - sg / K);
          if (!(fe[0] > T(0))) ev = T(1);
        }
        if (caps) atomicAdd(&I.stats->rootfind_cap_hits, (unsigned long long)caps);
        if (iters) atomicMax(&I.stats->rootfind_max_iters, (unsigned int)iters);
      }
      block_max_atomic(v, &I.stats->max_bound_violation);
      block_max_atomic(ev, &I.stats->max_entropy_violation);
    }
  } else if (act) {
#pragma unroll
    for (int f = 0; f < NC; ++f) fe[f] = (A.limiter == 0) ? uH[f] : uL[f];
  }
  if (act) {
    if (!move) {
#pragma unroll
      for (int f = 0; f < NC; ++f) fe[f] = u[f];
    }
#pragma unroll
    for (int f = 0; f < NC; ++f) {
      const T v = (I.c0 == T(0)) ? fe[f] : I.c0 * I.u0[f * N + g] + I.c1 * fe[f];
      I.uout[f * N + g] = v;
    }
  }
}

// CFL bound of Eq. cfl-low per node: m_i / (2 sum_{j != i} d-hat_ij); min-reduced into *out_bits
// (positive doubles order like their bit patterns).
template <int P, class LAW, typename T>
__global__ void __launch_bounds__(256) k_dt(const StageLaunch<T> A, unsigned long long* out_bits) {
  constexpr int n = P + 1, NN = n * n, NC = LAW::NC;
  using Aux = typename LAW::Aux;
  const Instance<T>& I = A.inst;
  const LawParams& lp = A.lp;
  const long long Ne = (long long)I.nx * I.ny;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double val = DBL_MAX;
  if (g < Ne * NN) {
    const long long e = g / NN;
    const int node = (int)(g - e * NN), a = node / n, b = node - a * n;
    const int ex = (int)(e % I.nx), ey = (int)(e / I.nx);
    const long long N = I.N;
    T u[NC], v[NC];
    Aux ax, av;
#pragma unroll
    for (int f = 0; f < NC; ++f) u[f] = I.uin[f * N + g];
    LAW::aux(u, ax, lp);
    T lam[4];
#pragma unroll
    for (int side = 0; side < 4; ++side) {
      const int k = side >> 1;
      const bool lower = (side & 1) == 0;
      const int idx = (k == 0) ? b : a;
      const bool inside = lower ? (idx > 0) : (idx < P);
      if (inside) {
        const long long gn = g + (k == 0 ? (lower ? -1 : 1) : (lower ? -n : n));
#pragma unroll
        for (int f = 0; f < NC; ++f) v[f] = I.uin[f * N + gn];
      } else {
        neighbor_state<P, NC>(I, side, e, ex, ey, (k == 0) ? a : b, u, v);
      }
      LAW::aux(v, av, lp);
      lam[side] = lower ? LAW::lam(k, v, av, u, ax, lp) : LAW::lam(k, u, ax, v, av, lp);
    }
    const double h = I.h;
    const double wa = (double)A.tab.w[a], wb = (double)A.tab.w[b];
    const double m = h * h * wa * wb;
    const double sumd = 0.5 * h * wa * ((double)lam[0] + (double)lam[1]) + 0.5 * h * wb * ((double)lam[2] + (double)lam[3]);
    if (sumd > 0.0) val = m / (2.0 * sumd);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x < 32) {
    val = (threadIdx.x < (blockDim.x + 31) / 32) ? red[threadIdx.x] : DBL_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, o));
    if (threadIdx.x == 0 && val < DBL_MAX) atomicMin(out_bits, (unsigned long long)__double_as_longlong(val));
  }
}

template <int P, class LAW, typename T>
cudaError_t launch_stage_p(const StageLaunch<T>& a, cudaStream_t s) {
  constexpr int EPB = epb_for(P);
  constexpr size_t smem = stage_smem_bytes<P, LAW, T>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_stage<P, LAW, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  const long long Ne = (long long)a.inst.nx * a.inst.ny;
  const long long blocks = (Ne + EPB - 1) / EPB;
  if (blocks <= 0) return cudaSuccess;
  k_stage<P, LAW, T><<<(unsigned)blocks, stage_threads(P), smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, class LAW, typename T>
cudaError_t launch_dt_p(const StageLaunch<T>& a, unsigned long long* bits, cudaStream_t s) {
  constexpr int NN = (P + 1) * (P + 1);
  const long long total = (long long)a.inst.nx * a.inst.ny * NN;
  const long long blocks = (total + 255) / 256;
  if (blocks <= 0) return cudaSuccess;
  k_dt<P, LAW, T><<<(unsigned)blocks, 256, 0, s>>>(a, bits);
  return cudaGetLastError();
}

#define SIDP_DISPATCH_P(FN, ...)                    \
  switch (p) {                                      \
    case 1: return FN<1, LAWT, T>(__VA_ARGS__);     \
    case 2: return FN<2, LAWT, T>(__VA_ARGS__);     \
    case 3: return FN<3, LAWT, T>(__VA_ARGS__);     \
    case 4: return FN<4, LAWT, T>(__VA_ARGS__);     \
    case 5: return FN<5, LAWT, T>(__VA_ARGS__);     \
    case 6: return FN<6, LAWT, T>(__VA_ARGS__);     \
    case 7: return FN<7, LAWT, T>(__VA_ARGS__);     \
    default: return cudaErrorInvalidValue;          \
  }

// Instantiate the launchers of one law and precision in the including translation unit.
#define SIDP_INSTANTIATE(LAWID, LAWTPL, TT)                                                          \
  template <>                                                                                        \
  cudaError_t launch_stage_law<LAWID, TT>(int p, const StageLaunch<TT>& a, cudaStream_t s) {        \
    using T = TT;                                                                                    \
    using LAWT = LAWTPL<TT>;                                                                         \
    SIDP_DISPATCH_P(launch_stage_p, a, s)                                                            \
  }                                                                                                  \
  template <>                                                                                        \
  cudaError_t launch_dt_law<LAWID, TT>(int p, const StageLaunch<TT>& a, unsigned long long* bits,   \
                                       cudaStream_t s) {                                             \
    using T = TT;                                                                                    \
    using LAWT = LAWTPL<TT>;                                                                         \
    SIDP_DISPATCH_P(launch_dt_p, a, bits, s)                                                         \
  }

}  // namespace sidp
