/*
 * potential.c -- shifted-force Lennard-Jones energy, forces and shear stress
 * of the oracle (FP64, all pairs).  Test infrastructure only; see oracle.h.
 *
 * Sec. 2.1: the energy landscape U(r) (Eq. 4) and the force f = -grad U
 * (Eq. 6).  Sec. 2.2, Eq. 13: LJ pair U(r) = 4 eps [(sig/r)^12 - (sig/r)^6].
 * The paper gives no cutoff; the workloads here use the shifted-force form
 *   U_sf(r) = U(r) - U(rc) - (r - rc) U'(rc)   for r < rc = rc_factor*sigma_ab
 * which makes energy and force continuous at rc.
 * Stress: tau = sigma_xy of Fig. 2(b), taken as (1/V) dE/dgamma along the
 * simple-shear affine path; per pair dr_x/dgamma = r_y, so
 *   tau = (1/V) sum_{i<j} U_sf'(r) d_x d_y / r.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double lj_u(double r, double sig, double eps) {
  double sr = sig / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
  return 4.0 * eps * (sr6 * sr6 - sr6);
}

static double lj_du(double r, double sig, double eps) {
  /* dU/dr = 4 eps (-12 sig^12 / r^13 + 6 sig^6 / r^7) */
  double sr = sig / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
  return -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
}

void orc_pair_sflj(double s, double sigma, double eps, double rc, double* u, double* du) {
  if (s >= rc * rc) {
    *u = 0.0;
    *du = 0.0;
    return;
  }
  double r = sqrt(s);
  double uc = lj_u(rc, sigma, eps), duc = lj_du(rc, sigma, eps);
  *u = lj_u(r, sigma, eps) - uc - (r - rc) * duc;
  *du = lj_du(r, sigma, eps) - duc;
}

int orc_energy_forces(const orc_potential* pot, int n, const double* x, const int32_t* types,
                      const double* H, double* E, double* F, double* tau) {
  int dim = pot->dim, nt = pot->n_types;
  double rcmax = 0.0;
  for (int k = 0; k < nt * nt; k++)
    if (pot->rc_factor * pot->sigma[k] > rcmax) rcmax = pot->rc_factor * pot->sigma[k];
  if (rcmax > orc_half_min_width(dim, H)) return ORC_ERR_BOX_TOO_SMALL;
  double e = 0.0, w = 0.0, d[3];
  if (F) memset(F, 0, sizeof(double) * (size_t)n * dim);
  for (int i = 0; i < n; i++) {
    for (int j = i + 1; j < n; j++) {
      /* d = r_j - r_i, minimum image */
      for (int c = 0; c < dim; c++) d[c] = x[j * dim + c] - x[i * dim + c];
      orc_min_image(dim, H, d);
      double s = 0.0;
      for (int c = 0; c < dim; c++) s += d[c] * d[c];
      int k = types[i] * nt + types[j];
      double rc = pot->rc_factor * pot->sigma[k];
      if (s >= rc * rc) continue;
      double u, du;
      orc_pair_sflj(s, pot->sigma[k], pot->eps[k], rc, &u, &du);
      double r = sqrt(s);
      e += u;
      /* force on i: -dU/dr_i = -U'(r) * (-d/r) = U'(r) d / r ; on j opposite */
      if (F)
        for (int c = 0; c < dim; c++) {
          F[i * dim + c] += du * d[c] / r;
          F[j * dim + c] -= du * d[c] / r;
        }
      w += du * d[0] * d[1] / r;
    }
  }
  *E = e;
  if (tau) *tau = w / orc_volume(dim, H);
  return ORC_OK;
}

double orc_fmax(int dim, int n, const double* F) {
  double m = 0.0;
  for (int i = 0; i < n; i++) {
    double s = 0.0;
    for (int c = 0; c < dim; c++) s += F[i * dim + c] * F[i * dim + c];
    if (!(s == s)) return NAN;
    if (s > m) m = s;
  }
  return sqrt(m);
}
