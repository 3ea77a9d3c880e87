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
//   lam_n(L, R, nx, ny) the same bound along a unit normal (nx, ny) (curved meshes)
//   limited field 0    (the scalar, or the density)
// Euler additionally: sigma = rho e / rho^gamma and psi_K(u) = rho e - K rho^gamma (Sec. 4.3).
#pragma once
#include <cmath>
#include "sidp_internal.h"

namespace sidp {

// min / max as single instructions (inputs are finite: states are validated on entry)
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

// Precision-specific arithmetic.  float64: IEEE operations (parity with the float64 oracle).
// float32 (the mixed path): hardware approximations (MUFU-based reciprocal, reciprocal square
// root and exp2/log2; a few ulp), whose effect is covered by the bound checks of the update.
__device__ __forceinline__ double ppow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float ppow(float x, float y) { return __powf(x, y); }
__device__ __forceinline__ double psqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float psqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double plog10(double x) { return log10(x); }
__device__ __forceinline__ float plog10(float x) { return log10f(x); }
__device__ __forceinline__ double psin(double x) { return sin(x); }
__device__ __forceinline__ float psin(float x) { return sinf(x); }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
// x^(2 gamma/(gamma-1)): seven multiplications' worth when the exponent is 7 (gamma = 1.4) in float32
__device__ __forceinline__ double pstar_pow(double x, const LawParamsT<double>& lp) { return pow(x, lp.inv_e); }
__device__ __forceinline__ float pstar_pow(float x, const LawParamsT<float>& lp) {
  if (lp.pow7) { const float x2 = x * x, x4 = x2 * x2; return x4 * x2 * x; }
  return __powf(x, lp.inv_e);
}

// Per-field arithmetic over the NC fields of a state.  sm_100 and later issue two float32
// operations per instruction on a register pair (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2); each
// lane is the correctly rounded scalar operation, so the pair forms equal a scalar loop whose
// products are contracted into fused multiply-adds.  Even field counts in float32 take the
// pairs; float64 and odd field counts the scalar loop.
template <int NC, typename T>
struct Pair {
  static constexpr bool on = sizeof(T) == 4 && NC % 2 == 0;
};

// d = s x + y
template <int NC, typename T>
__device__ __forceinline__ void v_fma(T* d, T s, const T* x, const T* y) {
  if constexpr (Pair<NC, T>::on) {
#pragma unroll
    for (int q = 0; q < NC; q += 2) {
      const float2 r = __ffma2_rn(make_float2(s, s), make_float2(x[q], x[q + 1]), make_float2(y[q], y[q + 1]));
      d[q] = r.x;
      d[q + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) d[q] = fma(s, x[q], y[q]);
  }
}

// d = x + y
template <int NC, typename T>
__device__ __forceinline__ void v_add(T* d, const T* x, const T* y) {
  if constexpr (Pair<NC, T>::on) {
#pragma unroll
    for (int q = 0; q < NC; q += 2) {
      const float2 r = __fadd2_rn(make_float2(x[q], x[q + 1]), make_float2(y[q], y[q + 1]));
      d[q] = r.x;
      d[q + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) d[q] = x[q] + y[q];
  }
}

// d = x - y
template <int NC, typename T>
__device__ __forceinline__ void v_sub(T* d, const T* x, const T* y) {
  if constexpr (Pair<NC, T>::on) {
#pragma unroll
    for (int q = 0; q < NC; q += 2) {
      const float2 r = __fadd2_rn(make_float2(x[q], x[q + 1]), make_float2(-y[q], -y[q + 1]));
      d[q] = r.x;
      d[q + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) d[q] = x[q] - y[q];
  }
}

// d = s x
template <int NC, typename T>
__device__ __forceinline__ void v_scale(T* d, T s, const T* x) {
  if constexpr (Pair<NC, T>::on) {
#pragma unroll
    for (int q = 0; q < NC; q += 2) {
      const float2 r = __fmul2_rn(make_float2(s, s), make_float2(x[q], x[q + 1]));
      d[q] = r.x;
      d[q + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) d[q] = s * x[q];
  }
}

template <typename T>
struct LawAdvection {
  static constexpr int NC = 1;
  static constexpr bool kEntropy = false;
  struct Aux {};
  __device__ static void aux(const T*, Aux&, const LawParamsT<T>&) {}
  __device__ static void flux(const T* u, const Aux&, int k, T* f, const LawParamsT<T>& lp) {
    f[0] = lp.beta[k] * u[0];
  }
  __device__ static T lam(int k, const T*, const Aux&, const T*, const Aux&, const LawParamsT<T>& lp) {
    return fabs(lp.beta[k]);
  }
  __device__ static T lam_n(const T*, const Aux&, const T*, const Aux&, T nx, T ny, const LawParamsT<T>& lp) {
    return fabs(lp.beta[0] * nx + lp.beta[1] * ny);
  }
};

// Linear advection with the divergence-free velocity beta = (b0x + bxy y, b0y + byx x) (Sec. 3.3):
// each component is constant along its own direction, so beta.n is continuous across every face,
// the discrete divergence sum_j c-hat_ij . beta_j vanishes, and the modified coefficients
// d-hat_ij = max(|c-hat_ij . beta_i|, |c-hat_ji . beta_j|) and bar states of Sec. 3.3 equal the
// face flux forms below.  The node's velocity is the law's per-node quantity (from its position).
template <typename T>
struct LawAdvectionVar {
  static constexpr int NC = 1;
  static constexpr bool kEntropy = false;
  static constexpr bool kPosition = true;
  struct Aux { T b[2]; };
  __device__ static void aux_at(const T*, T x, T y, Aux& a, const LawParamsT<T>& lp) {
    a.b[0] = lp.beta[0] + lp.bxy * y;
    a.b[1] = lp.beta[1] + lp.byx * x;
  }
  __device__ static void aux(const T*, Aux&, const LawParamsT<T>&) {}
  __device__ static void flux(const T* u, const Aux& a, int k, T* f, const LawParamsT<T>&) { f[0] = a.b[k] * u[0]; }
  __device__ static T lam(int k, const T*, const Aux& L, const T*, const Aux& R, const LawParamsT<T>&) {
    return tmax(fabs(L.b[k]), fabs(R.b[k]));
  }
};

template <typename T>
struct LawBurgers {
  static constexpr int NC = 1;
  static constexpr bool kEntropy = false;
  struct Aux {};
  __device__ static void aux(const T*, Aux&, const LawParamsT<T>&) {}
  __device__ static void flux(const T* u, const Aux&, int, T* f, const LawParamsT<T>&) {
    f[0] = T(0.5) * u[0] * u[0];
  }
  // F.e_k = u^2/2 is convex; the extreme characteristic speeds are the end states'.
  __device__ static T lam(int, const T* uL, const Aux&, const T* uR, const Aux&, const LawParamsT<T>&) {
    return tmax(fabs(uL[0]), fabs(uR[0]));
  }
  // F.n = (nx + ny) u^2/2: speed (nx + ny) u, extreme at an end state
  __device__ static T lam_n(const T* uL, const Aux&, const T* uR, const Aux&, T nx, T ny, const LawParamsT<T>&) {
    return fabs(nx + ny) * tmax(fabs(uL[0]), fabs(uR[0]));
  }
};

template <typename T>
struct LawEuler {
  static constexpr int NC = 4;
  static constexpr bool kEntropy = true;
  // Per-node quantities kept for the faces (16 bytes in float32): the normal velocity is
  // m_k / rho, and the two-rarefaction bound needs p only through p*/p.
  struct alignas(4 * sizeof(T) >= 16 ? 16 : 4 * sizeof(T)) Aux {
    T rinv;   // 1 / rho
    T a;      // sound speed
    T apm;    // a p^{-(gamma-1)/(2 gamma)}
    T ip;     // 1 / p
  };
  // Pressure (Eq. euler-eos), aux, and both flux components (Eq. euler-flux) of one node.
  __device__ static T pressure(const T* u, T rinv, const LawParamsT<T>& lp) {
    return lp.gm1 * (u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) * rinv);
  }
  __device__ static void aux(const T* u, Aux& x, const LawParamsT<T>& lp) {
    x.rinv = frcp(u[0]);
    const T p = pressure(u, x.rinv, lp);
    x.a = psqrt(lp.gamma * p * x.rinv);
    x.ip = frcp(p);
    x.apm = x.a * ppow(p, lp.neg_e);
  }
  // Eq. euler-flux along e_k: (m_k, m_k v_x + p d_{0k}, m_k v_y + p d_{1k}, (rho E + p) v_k)
  __device__ static void flux(const T* u, const Aux& x, int k, T* f, const LawParamsT<T>& lp) {
    const T p = pressure(u, x.rinv, lp);
    const T mk = u[1 + k];
    const T vk = mk * x.rinv;
    f[0] = mk;
    f[1] = u[1] * vk + (k == 0 ? p : T(0));
    f[2] = u[2] * vk + (k == 1 ? p : T(0));
    f[3] = (u[3] + p) * vk;
  }
  // Guermond-Popov two-rarefaction bound (guaranteed for 1 < gamma <= 5/3): the two-rarefaction
  // pressure p* bounds the star pressure from above, and the extreme speeds grow with it.
  __device__ static T lam(int k, const T* uL, const Aux& L, const T* uR, const Aux& R, const LawParamsT<T>& lp) {
    const T vL = uL[1 + k] * L.rinv, vR = uR[1 + k] * R.rinv;
    const T num = tmax(L.a + R.a - lp.half_gm1 * (vR - vL), T(0));
    const T ps = pstar_pow(fdiv(num, L.apm + R.apm), lp);
    const T lL = vL - L.a * psqrt(T(1) + lp.c_gp * tmax(ps * L.ip - T(1), T(0)));
    const T lR = vR + R.a * psqrt(T(1) + lp.c_gp * tmax(ps * R.ip - T(1), T(0)));
    return tmax(fabs(lL), fabs(lR));
  }
  // the same bound along the unit normal (nx, ny): normal velocities m.n / rho
  __device__ static T lam_n(const T* uL, const Aux& L, const T* uR, const Aux& R, T nx, T ny, const LawParamsT<T>& lp) {
    const T vL = (uL[1] * nx + uL[2] * ny) * L.rinv, vR = (uR[1] * nx + uR[2] * ny) * R.rinv;
    const T num = tmax(L.a + R.a - lp.half_gm1 * (vR - vL), T(0));
    const T ps = pstar_pow(fdiv(num, L.apm + R.apm), lp);
    const T lL = vL - L.a * psqrt(T(1) + lp.c_gp * tmax(ps * L.ip - T(1), T(0)));
    const T lR = vR + R.a * psqrt(T(1) + lp.c_gp * tmax(ps * R.ip - T(1), T(0)));
    return tmax(fabs(lL), fabs(lR));
  }
  // Internal energy rho e = rho E - |m|^2 / (2 rho).  Where kinetic energy dominates, the
  // subtraction cancels; the float32 path therefore carries the rounding errors of |m|^2 and of
  // the division (exact via fma) so that rho e keeps a relative error of a few ulp.
  __device__ static T rhoe(const T* u) {
    if constexpr (sizeof(T) == 8) {
      return u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0];
    } else {
      const float a = u[1] * u[1], ea = fmaf(u[1], u[1], -a);
      const float b = u[2] * u[2], eb = fmaf(u[2], u[2], -b);
      const float s = a + b, bb = s - a, es = (a - (s - bb)) + (b - bb);
      const float rinv = frcp(u[0]);
      const float q = s * rinv;                                  // |m|^2 / rho, rounded
      const float dq = (fmaf(-q, u[0], s) + (es + ea + eb)) * rinv;  // its correction
      return (u[3] - 0.5f * q) - 0.5f * dq;
    }
  }
  // sigma = rho e rho^-gamma; s = log(sigma)/(gamma-1) (Sec. 4.3)
  __device__ static T sigma(const T* u, const Aux&, const LawParamsT<T>& lp) { return rhoe(u) * ppow(u[0], -lp.gamma); }
  __device__ static T sigma_of(const T* u, const LawParamsT<T>& lp) { return rhoe(u) * ppow(u[0], -lp.gamma); }
  // psi_K(u) = rho e - K rho^gamma and its gradient in conserved variables
  __device__ static T psi(const T* u, T K, const LawParamsT<T>& lp) { return rhoe(u) - K * ppow(u[0], lp.gamma); }
  // True when psi_K(u) >= target is certain from a cheap float32 evaluation: the few roundings
  // of rho E and |m|^2/(2 rho) stay below 1e-6 of their magnitudes (a wide margin over the ~10
  // ulp they can reach), and K rho^gamma below 4e-6 of its (the fast power's relative error grows
  // with |gamma log2 rho|: about 1.9e-6 at gamma = 1.4 for rho = 256 or 1/256), so psi >=
  // psi_fast - err.  False means "undecided" (the caller evaluates psi in full).  The float64
  // path always evaluates psi.
  __device__ static bool psi_certainly_ge(const T* u, T K, T target, const LawParamsT<T>& lp) {
    if constexpr (sizeof(T) == 8) {
      return false;
    } else {
      const float rinv = frcp(u[0]);
      const float ke = 0.5f * fmaf(u[1], u[1], u[2] * u[2]) * rinv;
      const float rg = K * ppow(u[0], lp.gamma);
      const float pf = (u[3] - ke) - rg;
      const float err = 1e-6f * (fabsf(u[3]) + ke) + 4e-6f * rg;
      return pf - err >= target;
    }
  }
  __device__ static T psi_grad_dot(const T* u, T K, const T* w, const LawParamsT<T>& lp) {
    const T rinv = frcp(u[0]);
    const T vx = u[1] * rinv, vy = u[2] * rinv;
    const T drho = T(0.5) * (vx * vx + vy * vy) - lp.gamma * K * ppow(u[0], lp.gm1);
    return drho * w[0] - vx * w[1] - vy * w[2] + w[3];
  }
};

}  // namespace sidp
