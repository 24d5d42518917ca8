/*
 * geometry.c -- cell, minimum image and affine maps of the oracle (FP64).
 * Test infrastructure only; see oracle.h.
 *
 * Sec. 2.1: the cell is the Bravais tensor H, deformation acts as
 * H^(g+dg) = F^(dg) H^(g) (Eq. 1) and on every atom as r_i -> F r_i
 * (Eqs. 2-3).  Simple shear is F = [[1, dg], [0, 1]] (Eq. 16), in 3D with the
 * same xy entry and an identity z row/column.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

double orc_volume(int dim, const double* H) {
  /* upper-triangular H: determinant is the product of the diagonal */
  double v = 1.0;
  for (int a = 0; a < dim; a++) v *= H[a * dim + a];
  return fabs(v);
}

void orc_min_image(int dim, const double* H, double* d) {
  /* H is upper triangular, so column c (Bravais vector h_c) only has
   * components 0..c.  Removing whole lattice vectors from the last axis to the
   * first fixes one fractional coordinate per step without disturbing the
   * ones already fixed. */
  for (int c = dim - 1; c >= 0; c--) {
    double n = round(d[c] / H[c * dim + c]);
    if (n != 0.0)
      for (int a = 0; a <= c; a++) d[a] -= n * H[a * dim + c];
  }
}

double orc_half_min_width(int dim, const double* H) {
  /* perpendicular width along axis c = V / |area of the face spanned by the
   * other Bravais vectors|; for the triangular cells used here:
   *   2D: w_x = Lx * Ly / |h2| ... computed generally from cross products. */
  double V = orc_volume(dim, H);
  double wmin = INFINITY;
  if (dim == 2) {
    for (int c = 0; c < 2; c++) {
      int o = 1 - c; /* the other vector */
      double len = hypot(H[0 * 2 + o], H[1 * 2 + o]);
      double w = V / len;
      if (w < wmin) wmin = w;
    }
  } else {
    for (int c = 0; c < 3; c++) {
      int p = (c + 1) % 3, q = (c + 2) % 3;
      double u[3] = {H[0 * 3 + p], H[1 * 3 + p], H[2 * 3 + p]};
      double v[3] = {H[0 * 3 + q], H[1 * 3 + q], H[2 * 3 + q]};
      double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
      double area = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      double w = V / area;
      if (w < wmin) wmin = w;
    }
  }
  return 0.5 * wmin;
}

void orc_affine_map(int dim, int n, double* x, double* H, const double* F) {
  double tmp[3];
  for (int i = 0; i < n; i++) {
    for (int a = 0; a < dim; a++) {
      double s = 0.0;
      for (int b = 0; b < dim; b++) s += F[a * dim + b] * x[i * dim + b];
      tmp[a] = s;
    }
    memcpy(&x[i * dim], tmp, sizeof(double) * dim);
  }
  double Hn[9];
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double s = 0.0;
      for (int b = 0; b < dim; b++) s += F[a * dim + b] * H[b * dim + c];
      Hn[a * dim + c] = s;
    }
  memcpy(H, Hn, sizeof(double) * dim * dim);
}

void orc_affine_shear(int dim, int n, double* x, double* H, double dgamma) {
  double F[9] = {0};
  for (int a = 0; a < dim; a++) F[a * dim + a] = 1.0;
  F[0 * dim + 1] = dgamma; /* Eq. 16: x += dgamma * y */
  orc_affine_map(dim, n, x, H, F);
}

void orc_triangularise(int dim, int n, double* x, double* H) {
  /* Gram-Schmidt on the Bravais vectors (columns of H): q_0 along h_0, q_1 the
   * part of h_1 orthogonal to q_0, q_2 = q_0 x q_1 (3D).  With Q = [q_0 q_1
   * q_2], R = Q^T H is upper triangular with a positive diagonal (det H > 0),
   * and x <- Q^T x rotates the configuration rigidly with the cell, which
   * leaves every pair distance and the energy unchanged. */
  double q[3][3] = {{0}}, h[3][3];
  for (int c = 0; c < dim; c++)
    for (int a = 0; a < dim; a++) h[c][a] = H[a * dim + c]; /* h[c] = column c */
  double l0 = 0.0;
  for (int a = 0; a < dim; a++) l0 += h[0][a] * h[0][a];
  l0 = sqrt(l0);
  for (int a = 0; a < dim; a++) q[0][a] = h[0][a] / l0;
  double p = 0.0;
  for (int a = 0; a < dim; a++) p += q[0][a] * h[1][a];
  double l1 = 0.0;
  for (int a = 0; a < dim; a++) {
    q[1][a] = h[1][a] - p * q[0][a];
    l1 += q[1][a] * q[1][a];
  }
  l1 = sqrt(l1);
  for (int a = 0; a < dim; a++) q[1][a] /= l1;
  if (dim == 3) {
    q[2][0] = q[0][1] * q[1][2] - q[0][2] * q[1][1];
    q[2][1] = q[0][2] * q[1][0] - q[0][0] * q[1][2];
    q[2][2] = q[0][0] * q[1][1] - q[0][1] * q[1][0];
  }
  double R[9];
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double v = 0.0;
      if (c >= a)
        for (int k = 0; k < dim; k++) v += q[a][k] * h[c][k];
      R[a * dim + c] = v;
    }
  for (int i = 0; i < n; i++) {
    double y[3];
    for (int a = 0; a < dim; a++) {
      double v = 0.0;
      for (int k = 0; k < dim; k++) v += q[a][k] * x[i * dim + k];
      y[a] = v;
    }
    for (int a = 0; a < dim; a++) x[i * dim + a] = y[a];
  }
  memcpy(H, R, sizeof(double) * dim * dim);
}

/* rows q[a] of the orthonormal frame Q of Gram-Schmidt on the columns of a
 * cell G (the frame in which G is upper triangular with a positive diagonal) */
static void gs_frame(int dim, const double* G, double q[3][3]) {
  double h[3][3];
  for (int c = 0; c < dim; c++)
    for (int a = 0; a < dim; a++) h[c][a] = G[a * dim + c];
  double l0 = 0.0;
  for (int a = 0; a < dim; a++) l0 += h[0][a] * h[0][a];
  l0 = sqrt(l0);
  for (int a = 0; a < dim; a++) q[0][a] = h[0][a] / l0;
  double p = 0.0;
  for (int a = 0; a < dim; a++) p += q[0][a] * h[1][a];
  double l1 = 0.0;
  for (int a = 0; a < dim; a++) {
    q[1][a] = h[1][a] - p * q[0][a];
    l1 += q[1][a] * q[1][a];
  }
  l1 = sqrt(l1);
  for (int a = 0; a < dim; a++) q[1][a] /= l1;
  if (dim == 3) {
    q[2][0] = q[0][1] * q[1][2] - q[0][2] * q[1][1];
    q[2][1] = q[0][2] * q[1][0] - q[0][0] * q[1][2];
    q[2][2] = q[0][0] * q[1][1] - q[0][1] * q[1][0];
  }
}

void orc_deform(int dim, int n, double* x, double* H, double* Hlab, const double* F) {
  /* The history acts on the laboratory cell, Hlab <- F Hlab (Eq. 1).  The
   * stored cell is its upper-triangular form R = Q^T Hlab (Q from
   * Gram-Schmidt), so the stored configuration is the laboratory one seen in
   * the frame Q.  One increment maps stored positions by
   *   M = Q_new^T F Q_old        (r_lab <- F r_lab, Eq. 3, in the two frames)
   * which is upper triangular, and sets H <- R_new.  For simple shear Q stays
   * the identity and M = F exactly. */
  double qo[3][3] = {{0}}, qn[3][3] = {{0}}, Hn[9], M[9], T[9];
  gs_frame(dim, Hlab, qo);
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double v = 0.0;
      for (int k = 0; k < dim; k++) v += F[a * dim + k] * Hlab[k * dim + c];
      Hn[a * dim + c] = v;
    }
  memcpy(Hlab, Hn, sizeof(double) * dim * dim);
  gs_frame(dim, Hlab, qn);
  /* T = F Q_old (columns of Q_old are the rows qo[.]), M = Q_new^T T */
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double v = 0.0;
      for (int k = 0; k < dim; k++) v += F[a * dim + k] * qo[c][k];
      T[a * dim + c] = v;
    }
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double v = 0.0;
      for (int k = 0; k < dim; k++) v += qn[a][k] * T[k * dim + c];
      M[a * dim + c] = c < a ? 0.0 : v;
    }
  double Hdummy[9];
  memcpy(Hdummy, H, sizeof(double) * dim * dim);
  orc_affine_map(dim, n, x, Hdummy, M);
  for (int a = 0; a < dim; a++)
    for (int c = 0; c < dim; c++) {
      double v = 0.0;
      if (c >= a)
        for (int k = 0; k < dim; k++) v += qn[a][k] * Hlab[k * dim + c];
      H[a * dim + c] = v;
    }
}

void orc_wrap(int dim, int n, double* x, const double* H) {
  /* fractional coordinates s = H^-1 r by back substitution (H upper
   * triangular), then r <- r - H floor(s) */
  for (int i = 0; i < n; i++) {
    double s[3], m[3];
    for (int c = dim - 1; c >= 0; c--) {
      double t = x[i * dim + c];
      for (int k = c + 1; k < dim; k++) t -= H[c * dim + k] * s[k];
      s[c] = t / H[c * dim + c];
    }
    for (int c = 0; c < dim; c++) m[c] = floor(s[c]);
    for (int a = 0; a < dim; a++)
      for (int c = a; c < dim; c++) x[i * dim + a] -= H[a * dim + c] * m[c];
  }
}

double orc_max_rel_disp(int dim, int n, const double* a, const double* b, const double* H) {
  /* u_i = mi(a_i - b_i); the minimum is degenerate under a uniform
   * translation, so the mean of u is removed before taking the largest norm. */
  double mean[3] = {0, 0, 0};
  double d[3];
  for (int i = 0; i < n; i++) {
    for (int c = 0; c < dim; c++) d[c] = a[i * dim + c] - b[i * dim + c];
    orc_min_image(dim, H, d);
    for (int c = 0; c < dim; c++) mean[c] += d[c];
  }
  for (int c = 0; c < dim; c++) mean[c] /= (double)n;
  double m = 0.0;
  for (int i = 0; i < n; i++) {
    double s = 0.0;
    for (int c = 0; c < dim; c++) d[c] = a[i * dim + c] - b[i * dim + c];
    orc_min_image(dim, H, d);
    for (int c = 0; c < dim; c++) s += (d[c] - mean[c]) * (d[c] - mean[c]);
    if (sqrt(s) > m) m = sqrt(s);
  }
  return m;
}
