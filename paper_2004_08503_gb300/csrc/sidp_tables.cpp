// Reference-element tables on the host, float64 (Sec. 2.1 nodal Gauss-Lobatto basis,
// Sec. 2.2 weighted differentiation matrix (D_1D)_ij = w_i phi_j'(xi_i)).
//
// Nodes: the p-1 interior Gauss-Lobatto points on [-1,1] are the roots of P_p'(x); they are
// found by Newton's method on q(x) = (1 - x^2) P_p'(x) started from the Chebyshev-Gauss-Lobatto
// points, with P_p and its derivatives from the three-term Legendre recurrence.  Weights:
// w_i = 2 / (p (p+1) P_p(x_i)^2).  Both are mapped to [0,1].
// Derivatives of the Lagrange basis: phi_j'(x_i) = prod_{k != j}(x_i - x_k) / prod_{k != j}(x_j - x_k)
// for i != j (the product formula), and phi_i'(x_i) = sum_{k != i} 1/(x_i - x_k).
#include <cmath>
#include "sidp_internal.h"

namespace sidp {

static void legendre(int p, double x, double* P, double* dP, double* d2P) {
  // P_k by recurrence; derivatives from (1-x^2) P_p' = p (P_{p-1} - x P_p) away from the ends.
  double pm1 = 1.0, pk = x;
  if (p == 0) { *P = 1.0; *dP = 0.0; *d2P = 0.0; return; }
  for (int k = 2; k <= p; ++k) {
    double pn = ((2.0 * k - 1.0) * x * pk - (k - 1.0) * pm1) / k;
    pm1 = pk;
    pk = pn;
  }
  *P = pk;
  double one_m_x2 = 1.0 - x * x;
  *dP = p * (pm1 - x * pk) / one_m_x2;
  // Legendre ODE: (1-x^2) P'' - 2x P' + p(p+1) P = 0
  *d2P = (2.0 * x * (*dP) - p * (p + 1.0) * pk) / one_m_x2;
}

void gll_tables(int p, double* xi, double* w, double* D) {
  const int n = p + 1;
  double x[kMaxN];
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(p, t, &P, &dP, &d2P);
      double dt = dP / d2P;  // Newton on P_p'
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[i] = t;
  }
  for (int i = 0; i < n; ++i) {
    // P_p at the node by the plain recurrence (valid at the end points too)
    double pm1 = 1.0, pk = x[i];
    for (int k = 2; k <= p; ++k) {
      double pn = ((2.0 * k - 1.0) * x[i] * pk - (k - 1.0) * pm1) / k;
      pm1 = pk;
      pk = pn;
    }
    double Pp = (p == 0) ? 1.0 : pk;
    w[i] = 0.5 * 2.0 / (p * (p + 1.0) * Pp * Pp);
    xi[i] = 0.5 * (x[i] + 1.0);
  }
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double d;
      if (i != j) {
        double num = 1.0, den = 1.0;
        for (int k = 0; k < n; ++k) {
          if (k == j) continue;
          den *= (xi[j] - xi[k]);
          if (k != i) num *= (xi[i] - xi[k]);
        }
        d = num / den;
      } else {
        d = 0.0;
        for (int k = 0; k < n; ++k)
          if (k != i) d += 1.0 / (xi[i] - xi[k]);
      }
      D[i * n + j] = w[i] * d;
    }
  }
}

// Nodal-to-modal transform of the Gauss-Lobatto interpolant: coefficients c_k of the Legendre
// polynomials L_k(2x-1) on [0,1].  The discrete Gram matrix sum_i w_i L_j(x_i) L_k(x_i) is diagonal
// on the Gauss-Lobatto nodes (exact quadrature up to degree 2p-1 for j != k), so
// Vinv[k][i] = w_i L_k(x_i) / gamma_k with gamma_k = sum_i w_i L_k(x_i)^2.  nrm[k] = 1/(2k+1) is
// the exact squared norm of L_k(2x-1) on [0,1].
void modal_tables(int p, double* Vinv, double* nrm) {
  const int n = p + 1;
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  gll_tables(p, xi, w, D);
  double L[kMaxN][kMaxN];  // L[k][i] = L_k(2 xi_i - 1)
  for (int i = 0; i < n; ++i) {
    const double x = 2.0 * xi[i] - 1.0;
    double lm1 = 1.0, l = x;
    L[0][i] = 1.0;
    if (p >= 1) L[1][i] = x;
    for (int k = 2; k <= p; ++k) {
      const double ln = ((2.0 * k - 1.0) * x * l - (k - 1.0) * lm1) / k;
      lm1 = l;
      l = ln;
      L[k][i] = l;
    }
  }
  for (int k = 0; k < n; ++k) {
    double g = 0.0;
    for (int i = 0; i < n; ++i) g += w[i] * L[k][i] * L[k][i];
    for (int i = 0; i < n; ++i) Vinv[k * n + i] = w[i] * L[k][i] / g;
    nrm[k] = 1.0 / (2.0 * k + 1.0);
  }
}

}  // namespace sidp
