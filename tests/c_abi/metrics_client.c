/* A plain C99 client of libsidp: includes the public header, computes the metric arrays of a
 * 2 x 2 mesh at p = 2 whose nodes are the Cartesian ones scaled by 2 in x and 3 in y (affine),
 * and prints checks that the mapping fixes: det J = 6 h^2 at every node (m_i = w_a w_b 6 h^2 sums
 * to the area 6), rows of G J^-1 = (3h, 0) and (0, 2h), and a status string.  Needs no GPU. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "sidp.h"

int main(void) {
  const int p = 2, nx = 2, ny = 2, n = p + 1, NN = n * n;
  const long long N = (long long)nx * ny * NN;
  const double xi[3] = {0.0, 0.5, 1.0}, h = 0.5;
  double* x = malloc(sizeof(double) * N);
  double* y = malloc(sizeof(double) * N);
  double* out = malloc(sizeof(double) * SIDP_GEO_FIELDS * N);
  const int bc[4] = {SIDP_BC_PERIODIC, SIDP_BC_PERIODIC, SIDP_BC_OUTFLOW, SIDP_BC_OUTFLOW};
  for (int e = 0; e < nx * ny; ++e)
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        const long long g = (long long)e * NN + a * n + b;
        x[g] = 2.0 * ((e % nx) + xi[b]) * h;
        y[g] = 3.0 * ((e / nx) + xi[a]) * h;
      }
  sidp_status st = sidp_curved_metrics(p, nx, ny, bc, x, y, out);
  if (st != SIDP_OK) { printf("status %s\n", sidp_status_str(st)); return 1; }
  double area = 0.0, err = 0.0;
  for (long long g = 0; g < N; ++g) {
    area += out[8 * N + g];
    err = fmax(err, fabs(out[0 * N + g] - 3.0 * h));   /* row 1 = (y_eta, -x_eta) */
    err = fmax(err, fabs(out[1 * N + g]));
    err = fmax(err, fabs(out[2 * N + g]));
    err = fmax(err, fabs(out[3 * N + g] - 2.0 * h));   /* row 2 = (-y_xi, x_xi) */
    err = fmax(err, fabs(out[4 * N + g] - out[0 * N + g]));  /* affine: no correction */
  }
  printf("area %.15f maxerr %.3e ok %s\n", area, err, sidp_status_str(SIDP_OK));
  /* an inverted map is rejected with an argument error */
  for (long long g = 0; g < N; ++g) x[g] = -x[g];
  st = sidp_curved_metrics(p, nx, ny, bc, x, y, out);
  printf("mirrored %s\n", sidp_status_str(st));
  free(x); free(y); free(out);
  return 0;
}
