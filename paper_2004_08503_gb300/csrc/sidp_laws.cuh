// Device-side physical laws (Sec. 2.1, Sec. 3.3, Sec. 4.3).
//
// Each law provides, for a stage precision T:
//   NC                 number of conserved fields
//   Aux                per-node quantities reused by every face the node touches
//   aux(u)             fill Aux from the conserved state
//   flux(u, aux, k)    k-th component of F(u) (k = 0: x, 1: y), all NC fields
//   lam(k, L, R)       upper bound of lambda_max for the Riemann problem with left state L,
//                      right state R along +e_k (Sec. 2.1.1); the same bound serves the LF flux,
//                      d_ij (Eq. dij), the bar states and the CFL condition
//   limited field 0    (the scalar, or the density)
// Euler additionally: sigma = rho e / rho^gamma and psi_K(u) = rho e - K rho^gamma (Sec. 4.3).
#pragma once
#include <cmath>
#include "sidp_internal.h"

namespace sidp {

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// pow for positive x, precision-specific
__device__ __forceinline__ double ppow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float ppow(float x, float y) { return __powf(x, y); }
__device__ __forceinline__ double psqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float psqrt(float x) { return sqrtf(x); }

template <typename T>
struct LawAdvection {
  static constexpr int NC = 1;
  static constexpr bool kEntropy = false;
  struct Aux {};
  __device__ static void aux(const T*, Aux&, const LawParams&) {}
  __device__ static void flux(const T* u, const Aux&, int k, T* f, const LawParams& lp) {
    f[0] = T(lp.beta[k]) * u[0];
  }
  __device__ static T lam(int k, const T*, const Aux&, const T*, const Aux&, const LawParams& lp) {
    return fabs(T(lp.beta[k]));
  }
};

template <typename T>
struct LawBurgers {
  static constexpr int NC = 1;
  static constexpr bool kEntropy = false;
  struct Aux {};
  __device__ static void aux(const T*, Aux&, const LawParams&) {}
  __device__ static void flux(const T* u, const Aux&, int, T* f, const LawParams&) {
    f[0] = T(0.5) * u[0] * u[0];
  }
  // F.e_k = u^2/2 is convex; the extreme characteristic speeds are the end states'.
  __device__ static T lam(int, const T* uL, const Aux&, const T* uR, const Aux&, const LawParams&) {
    return tmax(fabs(uL[0]), fabs(uR[0]));
  }
};

template <typename T>
struct LawEuler {
  static constexpr int NC = 4;
  static constexpr bool kEntropy = true;
  struct Aux {
    T v[2];   // velocity
    T p;      // pressure
    T a;      // sound speed
    T pm;     // p^{-(gamma-1)/(2 gamma)}
  };
  __device__ static void aux(const T* u, Aux& x, const LawParams& lp) {
    const T g = T(lp.gamma);
    const T rinv = T(1) / u[0];
    x.v[0] = u[1] * rinv;
    x.v[1] = u[2] * rinv;
    x.p = (g - T(1)) * (u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) * rinv);  // Eq. euler-eos
    x.a = psqrt(g * x.p * rinv);
    x.pm = ppow(x.p, -(g - T(1)) / (T(2) * g));
  }
  // Eq. euler-flux along e_k: (m_k, m_k v_x + p d_{0k}, m_k v_y + p d_{1k}, (rho E + p) v_k)
  __device__ static void flux(const T* u, const Aux& x, int k, T* f, const LawParams&) {
    const T mk = u[1 + k];
    f[0] = mk;
    f[1] = mk * x.v[0] + (k == 0 ? x.p : T(0));
    f[2] = mk * x.v[1] + (k == 1 ? x.p : T(0));
    f[3] = (u[3] + x.p) * x.v[k];
  }
  // Guermond-Popov two-rarefaction bound (guaranteed for 1 < gamma <= 5/3): the two-rarefaction
  // pressure bounds the star pressure from above, and the extreme speeds grow with it.
  __device__ static T lam(int k, const T*, const Aux& L, const T*, const Aux& R, const LawParams& lp) {
    const T g = T(lp.gamma);
    const T e = (g - T(1)) / (T(2) * g);
    const T num = tmax(L.a + R.a - T(0.5) * (g - T(1)) * (R.v[k] - L.v[k]), T(0));
    const T den = L.a * L.pm + R.a * R.pm;
    const T ps = ppow(num / den, T(1) / e);
    const T c = (g + T(1)) / (T(2) * g);
    const T lL = L.v[k] - L.a * psqrt(T(1) + c * tmax(ps - L.p, T(0)) / L.p);
    const T lR = R.v[k] + R.a * psqrt(T(1) + c * tmax(ps - R.p, T(0)) / R.p);
    return tmax(fabs(lL), fabs(lR));
  }
  // sigma = rho e rho^-gamma; s = log(sigma)/(gamma-1) (Sec. 4.3)
  __device__ static T sigma(const T* u, const Aux& x, const LawParams& lp) {
    const T g = T(lp.gamma);
    return x.p / (g - T(1)) * ppow(u[0], -g);
  }
  __device__ static T sigma_of(const T* u, const LawParams& lp) {
    const T g = T(lp.gamma);
    const T rhoe = u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0];
    return rhoe * ppow(u[0], -g);
  }
  // psi_K(u) = rho e - K rho^gamma and its gradient in conserved variables
  __device__ static T psi(const T* u, T K, const LawParams& lp) {
    const T g = T(lp.gamma);
    return u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0] - K * ppow(u[0], g);
  }
  __device__ static T psi_grad_dot(const T* u, T K, const T* w, const LawParams& lp) {
    const T g = T(lp.gamma);
    const T rinv = T(1) / u[0];
    const T vx = u[1] * rinv, vy = u[2] * rinv;
    const T drho = T(0.5) * (vx * vx + vy * vy) - g * K * ppow(u[0], g - T(1));
    return drho * w[0] - vx * w[1] - vy * w[2] + w[3];
  }
};

}  // namespace sidp
