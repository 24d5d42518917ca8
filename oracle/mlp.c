/*
 * mlp.c -- per-atom neighbour-shell features and the FP64 multilayer
 * perceptron of the learned warm start.  Test infrastructure only; see
 * oracle.h.
 *
 * The paper only names extrapolation of the minimiser's starting point as
 * future work (Sec. 5).  The warm start predicts the non-affine displacement
 * of the next strain increment per atom from the displacements to its nearest
 * neighbours; FIRE then finishes from that start.  This file is the plain
 * definition of the features and of the network (forward, loss, gradients).
 *
 * GELU(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2)), exact form.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
  double s;
  int j;
} cand;

static int cand_cmp(const void* a, const void* b) {
  const cand* x = (const cand*)a;
  const cand* y = (const cand*)b;
  if (x->s < y->s) return -1;
  if (x->s > y->s) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

int orc_knn_features(int dim, int n, const double* x, const int32_t* types, const double* H,
                     int n_types, int n_nb, double* feat) {
  if (n_nb > n - 1) return ORC_ERR_INVALID_ARG;
  int width = n_nb * dim + n_types;
  cand* c = malloc(sizeof(cand) * (size_t)n);
  double d[3];
  for (int i = 0; i < n; i++) {
    int m = 0;
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      double s = 0.0;
      for (int a = 0; a < dim; a++) d[a] = x[j * dim + a] - x[i * dim + a];
      orc_min_image(dim, H, d);
      for (int a = 0; a < dim; a++) s += d[a] * d[a];
      c[m].s = s;
      c[m].j = j;
      m++;
    }
    qsort(c, (size_t)m, sizeof(cand), cand_cmp);
    double* f = feat + (size_t)i * width;
    for (int k = 0; k < n_nb; k++) {
      int j = c[k].j;
      for (int a = 0; a < dim; a++) d[a] = x[j * dim + a] - x[i * dim + a];
      orc_min_image(dim, H, d);
      for (int a = 0; a < dim; a++) f[k * dim + a] = d[a];
    }
    for (int t = 0; t < n_types; t++) f[n_nb * dim + t] = (types[i] == t) ? 1.0 : 0.0;
  }
  free(c);
  return ORC_OK;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

static double gelu_grad(double z) {
  return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
}

/* forward pass keeping pre-activations Z_l and activations A_l (A_0 = X) */
static void forward_keep(int L, const int32_t* w, const double* const* W, const double* const* b,
                         int64_t m, const double* X, double** Z, double** A) {
  memcpy(A[0], X, sizeof(double) * (size_t)m * w[0]);
  for (int l = 0; l < L; l++) {
    int fi = w[l], fo = w[l + 1];
    for (int64_t r = 0; r < m; r++)
      for (int o = 0; o < fo; o++) {
        double s = b[l][o];
        for (int k = 0; k < fi; k++) s += W[l][(size_t)o * fi + k] * A[l][(size_t)r * fi + k];
        Z[l][(size_t)r * fo + o] = s;
        A[l + 1][(size_t)r * fo + o] = (l + 1 < L) ? gelu(s) : s;
      }
  }
}

static void alloc_acts(int L, const int32_t* w, int64_t m, double*** Z, double*** A) {
  *Z = malloc(sizeof(double*) * L);
  *A = malloc(sizeof(double*) * (L + 1));
  (*A)[0] = malloc(sizeof(double) * (size_t)m * w[0]);
  for (int l = 0; l < L; l++) {
    (*Z)[l] = malloc(sizeof(double) * (size_t)m * w[l + 1]);
    (*A)[l + 1] = malloc(sizeof(double) * (size_t)m * w[l + 1]);
  }
}

static void free_acts(int L, double** Z, double** A) {
  for (int l = 0; l < L; l++) {
    free(Z[l]);
    free(A[l + 1]);
  }
  free(A[0]);
  free(Z);
  free(A);
}

int orc_mlp_forward(int n_layers, const int32_t* width, const double* const* W,
                    const double* const* b, int64_t m, const double* X, double* Y) {
  double **Z, **A;
  alloc_acts(n_layers, width, m, &Z, &A);
  forward_keep(n_layers, width, W, b, m, X, Z, A);
  memcpy(Y, A[n_layers], sizeof(double) * (size_t)m * width[n_layers]);
  free_acts(n_layers, Z, A);
  return ORC_OK;
}

double orc_mlp_loss_grad(int n_layers, const int32_t* width, const double* const* W,
                         const double* const* b, int64_t m, const double* X, const double* T,
                         double* const* dW, double* const* db) {
  int L = n_layers;
  double **Z, **A;
  alloc_acts(L, width, m, &Z, &A);
  forward_keep(L, width, W, b, m, X, Z, A);
  int fo = width[L];
  /* loss = 0.5/m sum_r sum_o (Y - T)^2 ; dLoss/dY = (Y - T)/m */
  double loss = 0.0;
  double* G = malloc(sizeof(double) * (size_t)m * fo);
  for (int64_t k = 0; k < m * fo; k++) {
    double e = A[L][k] - T[k];
    loss += 0.5 * e * e;
    G[k] = e / (double)m;
  }
  loss /= (double)m;
  /* G holds dLoss/dZ_l for the current layer (output layer is linear) */
  for (int l = L - 1; l >= 0; l--) {
    int fi = width[l], fo_l = width[l + 1];
    for (int o = 0; o < fo_l; o++) {
      double sb = 0.0;
      for (int64_t r = 0; r < m; r++) sb += G[(size_t)r * fo_l + o];
      db[l][o] = sb;
      for (int k = 0; k < fi; k++) {
        double s = 0.0;
        for (int64_t r = 0; r < m; r++) s += G[(size_t)r * fo_l + o] * A[l][(size_t)r * fi + k];
        dW[l][(size_t)o * fi + k] = s;
      }
    }
    if (l > 0) {
      double* Gp = malloc(sizeof(double) * (size_t)m * fi);
      for (int64_t r = 0; r < m; r++)
        for (int k = 0; k < fi; k++) {
          double s = 0.0;
          for (int o = 0; o < fo_l; o++) s += G[(size_t)r * fo_l + o] * W[l][(size_t)o * fi + k];
          Gp[(size_t)r * fi + k] = s * gelu_grad(Z[l - 1][(size_t)r * fi + k]);
        }
      free(G);
      G = Gp;
    }
  }
  free(G);
  free_acts(L, Z, A);
  return loss;
}
