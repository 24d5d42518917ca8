/*
 * minimize.c -- the minimisation operator F: r -> r_inf of Sec. 2.1 (Eq. 10)
 * in the oracle: FIRE (the accelerated path's minimiser) and the paper's own
 * conjugate gradients.  Test infrastructure only; see oracle.h.
 *
 * FIRE as used here (the paper does not describe FIRE; this is the reading
 * shared with the library by specification):
 *   v = 0, dt = dt0, alpha = alpha0, npos = 0
 *   for it = 0, 1, ...
 *     F = force(x); fmax = max_a |F_a|
 *     stop (converged) if fmax < tol          -- tested before moving
 *     stop (not converged) if it == max_iter
 *     P = F . v                               (all dN components)
 *     if P >= 0: npos += 1; if npos > n_min: dt = min(dt f_inc, dt_max), alpha *= f_alpha
 *     else:      npos = 0; dt = max(dt f_dec, dt_min); alpha = alpha0; v = 0
 *     v += dt F                               (unit masses, semi-implicit Euler)
 *     v = (1 - alpha) v + alpha |v| / |F| F   (global norms)
 *     per atom: s_a = dt v_a; if |s_a| > max_step: s_a *= max_step / |s_a|
 *     x += s
 * P = 0 happens only at it = 0 (v = 0) and counts as "not uphill", so a fresh
 * minimisation starts at dt0.  The displacement cap acts per atom.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

int orc_fire(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
             const int32_t* types, const double* H, int64_t* iters, double* E, double* fmax_out,
             double* e_trace, uint8_t* reset_trace, int64_t trace_cap) {
  int dim = pot->dim;
  size_t nd = (size_t)n * dim;
  double* v = calloc(nd, sizeof(double));
  double* F = malloc(nd * sizeof(double));
  double dt = fp->dt0, alpha = fp->alpha0, e = 0.0, fm = 0.0;
  int npos = 0, status = ORC_ERR_NOT_CONVERGED;
  int64_t it;
  for (it = 0;; it++) {
    int st = orc_energy_forces(pot, n, x, types, H, &e, F, NULL);
    if (st != ORC_OK) {
      status = st;
      break;
    }
    fm = orc_fmax(dim, n, F);
    if (e_trace && it < trace_cap) e_trace[it] = e;
    if (!isfinite(fm) || !isfinite(e)) {
      status = ORC_ERR_NONFINITE;
      break;
    }
    if (fm < fp->tol) {
      status = ORC_OK;
      break;
    }
    if (it >= fp->max_iter) break;
    double P = 0.0;
    for (size_t k = 0; k < nd; k++) P += F[k] * v[k];
    int reset = 0;
    if (P >= 0.0) {
      npos++;
      if (npos > fp->n_min) {
        dt = fmin(dt * fp->f_inc, fp->dt_max);
        alpha *= fp->f_alpha;
      }
    } else {
      npos = 0;
      dt = fmax(dt * fp->f_dec, fp->dt_min);
      alpha = fp->alpha0;
      memset(v, 0, nd * sizeof(double));
      reset = 1;
    }
    if (reset_trace && it < trace_cap) reset_trace[it] = (uint8_t)reset;
    for (size_t k = 0; k < nd; k++) v[k] += dt * F[k];
    double vn = 0.0, fn = 0.0;
    for (size_t k = 0; k < nd; k++) {
      vn += v[k] * v[k];
      fn += F[k] * F[k];
    }
    vn = sqrt(vn);
    fn = sqrt(fn);
    for (size_t k = 0; k < nd; k++) v[k] = (1.0 - alpha) * v[k] + alpha * (vn / fn) * F[k];
    for (int i = 0; i < n; i++) {
      double s[3], len = 0.0;
      for (int c = 0; c < dim; c++) {
        s[c] = dt * v[i * dim + c];
        len += s[c] * s[c];
      }
      len = sqrt(len);
      double scale = len > fp->max_step ? fp->max_step / len : 1.0;
      for (int c = 0; c < dim; c++) x[i * dim + c] += scale * s[c];
    }
  }
  *iters = it;
  *E = e;
  *fmax_out = fm;
  free(v);
  free(F);
  return status;
}

/* Polak-Ribiere (non-negative beta) conjugate gradients with an Armijo
 * backtracking line search.  Every accepted step lowers the energy, so the
 * energy trace is strictly decreasing. */
int orc_cg(const orc_potential* pot, int n, double* x, const int32_t* types, const double* H,
           double tol, int64_t max_iter, int64_t* iters, double* E, double* fmax_out,
           double* e_trace, int64_t trace_cap) {
  int dim = pot->dim;
  size_t nd = (size_t)n * dim;
  double* F = malloc(nd * sizeof(double));
  double* Fn = malloc(nd * sizeof(double));
  double* d = malloc(nd * sizeof(double));
  double* xt = malloc(nd * sizeof(double));
  double e, et, fm;
  int status = ORC_ERR_NOT_CONVERGED;
  int st = orc_energy_forces(pot, n, x, types, H, &e, F, NULL);
  if (st != ORC_OK) {
    free(F); free(Fn); free(d); free(xt);
    return st;
  }
  memcpy(d, F, nd * sizeof(double));
  double step = 1e-3;
  int64_t it;
  for (it = 0;; it++) {
    fm = orc_fmax(dim, n, F);
    if (e_trace && it < trace_cap) e_trace[it] = e;
    if (!isfinite(fm)) {
      status = ORC_ERR_NONFINITE;
      break;
    }
    if (fm < tol) {
      status = ORC_OK;
      break;
    }
    if (it >= max_iter) break;
    /* descent direction: d . grad = -d . F must be negative */
    double slope = 0.0;
    for (size_t k = 0; k < nd; k++) slope -= d[k] * F[k];
    if (slope >= 0.0) {
      memcpy(d, F, nd * sizeof(double));
      slope = 0.0;
      for (size_t k = 0; k < nd; k++) slope -= d[k] * F[k];
    }
    double dmax = 0.0;
    for (int i = 0; i < n; i++) {
      double s = 0.0;
      for (int c = 0; c < dim; c++) s += d[i * dim + c] * d[i * dim + c];
      if (s > dmax) dmax = s;
    }
    dmax = sqrt(dmax);
    double a = fmin(2.0 * step, 0.1 / dmax);
    int accepted = 0;
    for (int bt = 0; bt < 200; bt++) {
      for (size_t k = 0; k < nd; k++) xt[k] = x[k] + a * d[k];
      orc_energy_forces(pot, n, xt, types, H, &et, Fn, NULL);
      if (et < e + 1e-4 * a * slope) {
        accepted = 1;
        break;
      }
      a *= 0.5;
    }
    if (!accepted) break; /* no further decrease representable */
    step = a;
    double num = 0.0, den = 0.0;
    for (size_t k = 0; k < nd; k++) {
      num += Fn[k] * (Fn[k] - F[k]);
      den += F[k] * F[k];
    }
    double beta = fmax(0.0, num / den);
    for (size_t k = 0; k < nd; k++) d[k] = Fn[k] + beta * d[k];
    memcpy(x, xt, nd * sizeof(double));
    memcpy(F, Fn, nd * sizeof(double));
    e = et;
  }
  *iters = it;
  *E = e;
  *fmax_out = fm;
  free(F); free(Fn); free(d); free(xt);
  return status;
}
