// Metric terms of curved (mapped) quadrilateral meshes, on the host in float64 (Sec. 2.3,
// Sec. 3.1).  Computed once per mesh by sidp_set_geometry (and exported on its own, so that the
// tables can be checked without a GPU); the stage and time-step kernels read the result.
//
// For element K with node coordinates (x, y) at the Gauss-Lobatto points, the reference
// derivatives of the interpolated map are taken with the nodal derivative matrix
// A_bc = phi_c'(xi_b) = D_bc / w_b.  Then G = det J = x_xi y_eta - x_eta y_xi and the rows of
// G J^-1 are row 1 = (y_eta, -x_eta), row 2 = (-y_xi, x_xi) (the two-dimensional cross-product
// form, which satisfies the metric identity Eq. metric exactly).
//
// Face normals: the normal of the face at node (a, 0) or (a, p), pointing in +xi, is row 1 there;
// two elements sharing a face (or a periodic side) use the mean of their two values, so the face
// has one normal; a face on a non-periodic boundary uses its own row.  Likewise +eta and row 2.
//
// Correction (Sec. 3.1): G J^-1-hat = G J^-1 + C with C the minimum-norm solution of
// Eq. metric-perturbation, A [C_1j; C_2j] = sum_e B_e n_{e,j} 1 - A [row1_j; row2_j],
// A = (D-hat_{1,R}^T  D-hat_{2,R}^T).  A has rank NN - 1 (its left null space is the constants),
// and the right-hand side sums to zero, so the minimum-norm solution is
// A^T (A A^T + 1 1^T / NN)^-1 rhs; the NN x NN matrix is inverted once per degree by Gauss-Jordan
// elimination with partial pivoting.
#include <cmath>
#include <vector>
#include "sidp_internal.h"

namespace sidp {

namespace {

// D-hat_1D of Eq. didp: row 0 (-1/2, 1/2), interior rows -1/2 at i-1 and +1/2 at i+1, last row
// (-1/2, 1/2) at (p-1, p).
double dhat(int n, int i, int j) {
  if (i == 0) return (j == 0) ? -0.5 : (j == 1) ? 0.5 : 0.0;
  if (i == n - 1) return (j == n - 2) ? -0.5 : (j == n - 1) ? 0.5 : 0.0;
  return (j == i - 1) ? -0.5 : (j == i + 1) ? 0.5 : 0.0;
}

// Minimum-norm solve operator P = A^T (A A^T + 1 1^T / NN)^-1, (2 NN) x NN, row-major.
bool min_norm_operator(int n, const double* w, std::vector<double>& P) {
  const int NN = n * n;
  // A[i][k] for k < NN: D-hat_{1,R}^T[i][k] = D-hat_{1,R}[k][i] = w_a' dhat(b', b) delta_{a a'}
  //          k >= NN:   D-hat_{2,R}^T[i][k-NN] = dhat(a', a) w_b' delta_{b b'}
  std::vector<double> A((size_t)NN * 2 * NN, 0.0);
  for (int i = 0; i < NN; ++i) {
    const int a = i / n, b = i % n;
    for (int k = 0; k < NN; ++k) {
      const int a2 = k / n, b2 = k % n;
      if (a2 == a) A[(size_t)i * 2 * NN + k] = w[a2] * dhat(n, b2, b);
      if (b2 == b) A[(size_t)i * 2 * NN + NN + k] = dhat(n, a2, a) * w[b2];
    }
  }
  // M = A A^T + 1 1^T / NN, augmented with the identity for Gauss-Jordan
  std::vector<double> M((size_t)NN * 2 * NN, 0.0);
  for (int i = 0; i < NN; ++i) {
    for (int j = 0; j < NN; ++j) {
      double s = 1.0 / NN;
      for (int k = 0; k < 2 * NN; ++k) s += A[(size_t)i * 2 * NN + k] * A[(size_t)j * 2 * NN + k];
      M[(size_t)i * 2 * NN + j] = s;
    }
    M[(size_t)i * 2 * NN + NN + i] = 1.0;
  }
  for (int c = 0; c < NN; ++c) {
    int piv = c;
    for (int r = c + 1; r < NN; ++r)
      if (std::fabs(M[(size_t)r * 2 * NN + c]) > std::fabs(M[(size_t)piv * 2 * NN + c])) piv = r;
    if (!(std::fabs(M[(size_t)piv * 2 * NN + c]) > 1e-300)) return false;
    if (piv != c)
      for (int k = 0; k < 2 * NN; ++k) std::swap(M[(size_t)c * 2 * NN + k], M[(size_t)piv * 2 * NN + k]);
    const double inv = 1.0 / M[(size_t)c * 2 * NN + c];
    for (int k = 0; k < 2 * NN; ++k) M[(size_t)c * 2 * NN + k] *= inv;
    for (int r = 0; r < NN; ++r) {
      if (r == c) continue;
      const double f = M[(size_t)r * 2 * NN + c];
      if (f == 0.0) continue;
      for (int k = 0; k < 2 * NN; ++k) M[(size_t)r * 2 * NN + k] -= f * M[(size_t)c * 2 * NN + k];
    }
  }
  // P[k][i] = sum_j A[j][k] Minv[j][i]
  P.assign((size_t)2 * NN * NN, 0.0);
  for (int k = 0; k < 2 * NN; ++k)
    for (int i = 0; i < NN; ++i) {
      double s = 0.0;
      for (int j = 0; j < NN; ++j) s += A[(size_t)j * 2 * NN + k] * M[(size_t)j * 2 * NN + NN + i];
      P[(size_t)k * NN + i] = s;
    }
  return true;
}

}  // namespace

sidp_status curved_metrics(int p, int nx, int ny, const int* bc, const double* x, const double* y, double* out,
                           std::string& msg) {
  if (p < 1 || p > kMaxP || nx < 1 || ny < 1 || !bc || !x || !y || !out) {
    msg = "curved metrics: invalid argument";
    return SIDP_ERR_ARG;
  }
  for (int s = 0; s < 4; ++s)
    if (bc[s] != SIDP_BC_PERIODIC && bc[s] != SIDP_BC_OUTFLOW && bc[s] != SIDP_BC_SLIP_WALL) {
      msg = "curved meshes take periodic, outflow or slip-wall sides";
      return SIDP_ERR_ARG;
    }
  const int n = p + 1, NN = n * n;
  const long long Ne = (long long)nx * ny, N = Ne * NN;
  double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
  gll_tables(p, xi, w, D);
  double Ad[kMaxN * kMaxN];
  for (int b = 0; b < n; ++b)
    for (int c = 0; c < n; ++c) Ad[b * n + c] = D[b * n + c] / w[b];
  std::vector<double> P;
  if (!min_norm_operator(n, w, P)) {
    msg = "curved metrics: singular reference matrix";
    return SIDP_ERR_ARG;
  }
  double* R1x = out + 0 * N; double* R1y = out + 1 * N;
  double* R2x = out + 2 * N; double* R2y = out + 3 * N;
  double* Q1x = out + 4 * N; double* Q1y = out + 5 * N;
  double* Q2x = out + 6 * N; double* Q2y = out + 7 * N;
  double* mass = out + 8 * N;
  double* NXx = out + 9 * N; double* NXy = out + 10 * N;
  double* NYx = out + 11 * N; double* NYy = out + 12 * N;
  // metric terms and masses
  // coordinates relative to the element's first node: the same map (derivatives of constants
  // vanish), differentiated without the cancellation of absolute coordinates (relative precision of
  // the derivatives independent of the element size)
  std::vector<double> xr(NN), yr(NN);
  for (long long e = 0; e < Ne; ++e) {
    const double* xe = x + e * NN;
    const double* ye = y + e * NN;
    for (int i = 0; i < NN; ++i) { xr[i] = xe[i] - xe[0]; yr[i] = ye[i] - ye[0]; }
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double x_xi = 0, y_xi = 0, x_eta = 0, y_eta = 0;
        for (int c = 0; c < n; ++c) {
          x_xi += Ad[b * n + c] * xr[a * n + c];
          y_xi += Ad[b * n + c] * yr[a * n + c];
          x_eta += Ad[a * n + c] * xr[c * n + b];
          y_eta += Ad[a * n + c] * yr[c * n + b];
        }
        const long long g = e * NN + a * n + b;
        const double G = x_xi * y_eta - x_eta * y_xi;
        if (!(G > 0.0) || !std::isfinite(G)) {
          msg = "curved metrics: det J <= 0 (or not finite) in element " + std::to_string(e);
          return SIDP_ERR_ARG;
        }
        R1x[g] = y_eta; R1y[g] = -x_eta;
        R2x[g] = -y_xi; R2y[g] = x_xi;
        mass[g] = w[a] * w[b] * G;
        NXx[g] = NXy[g] = NYx[g] = NYy[g] = 0.0;
      }
  }
  // face normals (+xi at b = 0, p; +eta at a = 0, p)
  for (long long e = 0; e < Ne; ++e) {
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    for (int side = 0; side < 4; ++side) {  // W, E, S, N
      const bool xface = side < 2;
      const bool lowside = (side == 0 || side == 2);
      int nex = ex, ney = ey;
      bool inside;
      if (side == 0) { nex = ex - 1; inside = ex > 0; }
      else if (side == 1) { nex = ex + 1; inside = ex < nx - 1; }
      else if (side == 2) { ney = ey - 1; inside = ey > 0; }
      else { ney = ey + 1; inside = ey < ny - 1; }
      const bool shared = inside || bc[side] == SIDP_BC_PERIODIC;
      const long long nb = (long long)((ney + ny) % ny) * nx + (nex + nx) % nx;
      for (int k = 0; k < n; ++k) {
        const int own = xface ? (k * n + (lowside ? 0 : p)) : ((lowside ? 0 : p) * n + k);
        const int opp = xface ? (k * n + (lowside ? p : 0)) : ((lowside ? p : 0) * n + k);
        const long long go = e * NN + own, gn = nb * NN + opp;
        const double* Rx = xface ? R1x : R2x;
        const double* Ry = xface ? R1y : R2y;
        double vx = Rx[go], vy = Ry[go];
        if (shared) {  // the low side's row plus the high side's row, halved (same order on both sides)
          const long long glo = lowside ? gn : go, ghi = lowside ? go : gn;
          vx = 0.5 * (Rx[glo] + Rx[ghi]);
          vy = 0.5 * (Ry[glo] + Ry[ghi]);
        }
        (xface ? NXx : NYx)[go] = vx;
        (xface ? NXy : NYy)[go] = vy;
      }
    }
  }
  // minimum-norm correction per element and component j
  std::vector<double> rhs(NN), sol(2 * NN);
  for (long long e = 0; e < Ne; ++e) {
    const long long g0 = e * NN;
    for (int j = 0; j < 2; ++j) {
      const double* r1 = (j == 0 ? R1x : R1y) + g0;
      const double* r2 = (j == 0 ? R2x : R2y) + g0;
      for (int i = 0; i < NN; ++i) {
        const int a = i / n, b = i % n;
        // sum_e B_e n_{e,j}: outward normals, face weight of the node along its face
        double bnd = 0.0;
        const double nxj = (j == 0 ? NXx : NXy)[g0 + i], nyj = (j == 0 ? NYx : NYy)[g0 + i];
        if (b == 0) bnd -= w[a] * nxj;
        if (b == p) bnd += w[a] * nxj;
        if (a == 0) bnd -= w[b] * nyj;
        if (a == p) bnd += w[b] * nyj;
        // (A [row1_j; row2_j])_i = sum_k D-hat_1[k][i] row1_j[k] + sum_k D-hat_2[k][i] row2_j[k]
        double av = 0.0;
        for (int c = 0; c < n; ++c) {
          av += w[a] * dhat(n, c, b) * r1[a * n + c];
          av += dhat(n, c, a) * w[b] * r2[c * n + b];
        }
        rhs[i] = bnd - av;
      }
      for (int k = 0; k < 2 * NN; ++k) {
        double s = 0.0;
        for (int i = 0; i < NN; ++i) s += P[(size_t)k * NN + i] * rhs[i];
        sol[k] = s;
      }
      double* q1 = (j == 0 ? Q1x : Q1y) + g0;
      double* q2 = (j == 0 ? Q2x : Q2y) + g0;
      for (int i = 0; i < NN; ++i) {
        q1[i] = r1[i] + sol[i];
        q2[i] = r2[i] + sol[NN + i];
      }
    }
  }
  return SIDP_OK;
}

}  // namespace sidp
