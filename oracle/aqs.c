/*
 * aqs.c -- the AQS protocol (Sec. 2.1, Eq. 12) and the two-level parallel
 * stepping scheme (Sec. 3, Algorithm 1) in the oracle.  Test infrastructure
 * only; see oracle.h.
 *
 * Readings where the paper is silent:
 *  - D_k, the non-affine displacement of step k, is
 *    max_a | mi(r_k,a - (F r_{k-1})_a) - mean |; a step is a plastic event when
 *    D_k exceeds a threshold chosen by the caller.
 *  - Equality of two minima (Eq. 20, same basin of Eq. 9) is decided by
 *    orc_max_rel_disp(in, out) < eq_tol: both are converged minima at the same
 *    strain, so equal basins give the same point up to the convergence
 *    tolerance, and different basins differ by a finite distance.
 *  - Last window: with rem = N_steps - N_current fine steps left, only
 *    P_eff = min(P, ceil(rem / K)) chains run, and when rem < P K the last one
 *    runs rem - (P_eff - 1) K steps, so the run ends exactly at N_steps.
 *  - q when P_eff = 1 (no equality test): the chain's own length.
 *  - On a failed test at chain i, r_star <- r_q with q = iK, which is the end
 *    of chain i-1 (the incoming configuration of the failed test).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* the deformation increment of step k: simple shear by dgamma (Eq. 16), or
 * the k-th matrix of a deformation history F (n_steps x d x d) */
static void increment(int dim, int n, double* x, double* H, double* Hlab, double dgamma,
                      const double* F, int k) {
  if (F) orc_deform(dim, n, x, H, Hlab, F + (size_t)k * dim * dim);
  else orc_affine_shear(dim, n, x, H, dgamma);
}

int orc_aqs_history(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
                    const int32_t* types, double* H, double* Hlab, double dgamma, const double* F,
                    int n_steps, double* E_k, double* tau_k, int64_t* iters_k, double* D_k) {
  int dim = pot->dim;
  if (F && !Hlab) return ORC_ERR_INVALID_ARG;
  size_t nd = (size_t)n * dim;
  double* xa = malloc(nd * sizeof(double));
  int status = ORC_OK;
  for (int k = 0; k < n_steps; k++) {
    increment(dim, n, x, H, Hlab, dgamma, F, k); /* F_N^(dgamma) r_{k-1} */
    memcpy(xa, x, nd * sizeof(double));
    int64_t it;
    double e, fm, tau;
    status = orc_fire(pot, fp, n, x, types, H, &it, &e, &fm, NULL, NULL, 0); /* F(.) */
    if (status != ORC_OK) break;
    orc_energy_forces(pot, n, x, types, H, &e, NULL, &tau);
    if (E_k) E_k[k] = e;
    if (tau_k) tau_k[k] = tau;
    if (iters_k) iters_k[k] = it;
    if (D_k) D_k[k] = orc_max_rel_disp(dim, n, x, xa, H);
  }
  free(xa);
  return status;
}

int orc_aqs(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
            const int32_t* types, double* H, double dgamma, int n_steps, double* E_k,
            double* tau_k, int64_t* iters_k, double* D_k) {
  return orc_aqs_history(pot, fp, n, x, types, H, NULL, dgamma, NULL, n_steps, E_k, tau_k,
                         iters_k, D_k);
}

int64_t orc_alg1_decide(int P_eff, const int32_t* K_i, const uint8_t* eq, int32_t* first_fail) {
  /* Algorithm 1: scan i = 1..P-1; an equal pair extends the accepted range to
   * the end of chain i, the first unequal pair stops the scan at its start. */
  int64_t q = K_i[0];
  *first_fail = -1;
  for (int i = 1; i < P_eff; i++) {
    if (eq[i]) {
      q += K_i[i];
    } else {
      *first_fail = i;
      break;
    }
  }
  return q;
}

/* one level-II chain: (F o F_N)^{K_i} o F applied to the level-I start */
typedef struct {
  const orc_potential* pot;
  const orc_fire_params* fp;
  int n;
  const int32_t* types;
  double dgamma;
  const double* F; /* the chain's fine increments (NULL: simple shear by dgamma) */
  int K_i;
  double* x;     /* in: level-I start; out: chain end */
  double* H;     /* in/out */
  double* Hlab;  /* in/out, laboratory cell (histories only) */
  double* x_out; /* out: F(start), the outgoing configuration */
  double* E, *tau, *D;
  int64_t* iters;
  int64_t iters_total;
  int status;
} chain_job;

static void* run_chain(void* arg) {
  chain_job* c = (chain_job*)arg;
  int dim = c->pot->dim;
  size_t nd = (size_t)c->n * dim;
  int64_t it;
  double e, fm;
  c->iters_total = 0;
  c->status = orc_fire(c->pot, c->fp, c->n, c->x, c->types, c->H, &it, &e, &fm, NULL, NULL, 0);
  c->iters_total += it;
  memcpy(c->x_out, c->x, nd * sizeof(double));
  if (c->status != ORC_OK) return NULL;
  c->status = orc_aqs_history(c->pot, c->fp, c->n, c->x, c->types, c->H, c->Hlab, c->dgamma,
                              c->F, c->K_i, c->E, c->tau, c->iters, c->D);
  for (int k = 0; k < c->K_i; k++) c->iters_total += c->iters[k];
  return NULL;
}

int orc_parallel(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
                 const int32_t* types, double* H, double dgamma, int K, int P, int n_steps,
                 double eq_tol, int n_threads, double* E_k, double* tau_k, int64_t* iters_k,
                 double* D_k, int64_t* log_iter, int32_t* log_i, uint8_t* log_eq, double* log_m,
                 int64_t log_cap, orc_parallel_stats* stats, int K_max, int32_t* K_pass,
                 int wrap_ends, const double* F_steps, double* Hlab) {
  if (K < 1 || P < 1 || n_steps < 0) return ORC_ERR_INVALID_ARG;
  if (F_steps && !Hlab) return ORC_ERR_INVALID_ARG;
  const int Kcap = K_max > K ? K_max : K; /* longest chain any pass can have */
  const int adaptive = K_max > K;
  int dim = pot->dim;
  size_t nd = (size_t)n * dim;
  double* xs = malloc(nd * sizeof(double) * P);   /* chain states */
  double* xo = malloc(nd * sizeof(double) * P);   /* outgoing configurations */
  double* Hs = malloc(sizeof(double) * 9 * P);  /* chain cells, sheared along the chain */
  double* H1 = malloc(sizeof(double) * 9 * P);  /* level-I cells: chain i starts at i dgamma^c */
  double* HL = malloc(sizeof(double) * 9 * P);  /* laboratory cells of the chains (histories) */
  double* cE = malloc(sizeof(double) * (size_t)Kcap * P);
  double* cT = malloc(sizeof(double) * (size_t)Kcap * P);
  double* cD = malloc(sizeof(double) * (size_t)Kcap * P);
  int64_t* cI = malloc(sizeof(int64_t) * (size_t)Kcap * P);
  chain_job* jobs = malloc(sizeof(chain_job) * P);
  pthread_t* th = malloc(sizeof(pthread_t) * P);
  int32_t* Ki = malloc(sizeof(int32_t) * P);
  uint8_t* eq = calloc(P, 1);
  int64_t n_cur = 0, iter = 0, n_log = 0, fire_total = 0;
  int status = ORC_OK;
  while (n_cur < n_steps) {
    double dgc = K * dgamma; /* coarse increment dgamma^c = K dgamma of this pass */
    if (K_pass) K_pass[iter] = K;
    int64_t rem = n_steps - n_cur;
    int P_eff = (int)((rem + K - 1) / K);
    if (P_eff > P) P_eff = P;
    for (int i = 0; i < P_eff; i++) Ki[i] = K;
    if (rem < (int64_t)P_eff * K) Ki[P_eff - 1] = (int32_t)(rem - (int64_t)(P_eff - 1) * K);
    /* level I: r^c_iK = F_N^(i dgamma^c) r_star (Sec. 3.2, Eq. 18).  With a
     * deformation history the coarse map is the product of the i K fine
     * increments that follow the current step, applied one after the other
     * (the sequence chain i-1 applies along its way), so that chain i starts
     * in exactly the cell in which chain i-1 ends. */
    for (int i = 0; i < P_eff; i++) {
      memcpy(xs + i * nd, x, nd * sizeof(double));
      memcpy(Hs + 9 * i, H, sizeof(double) * dim * dim);
      if (F_steps) {
        memcpy(HL + 9 * i, Hlab, sizeof(double) * dim * dim);
        for (int s = 0; s < i * K; s++)
          orc_deform(dim, n, xs + i * nd, Hs + 9 * i, HL + 9 * i,
                     F_steps + (size_t)(n_cur + s) * dim * dim);
      } else {
        orc_affine_shear(dim, n, xs + i * nd, Hs + 9 * i, i * dgc);
      }
      memcpy(H1 + 9 * i, Hs + 9 * i, sizeof(double) * dim * dim);
      chain_job* c = &jobs[i];
      c->pot = pot; c->fp = fp; c->n = n; c->types = types; c->dgamma = dgamma;
      c->K_i = Ki[i]; c->x = xs + i * nd; c->H = Hs + 9 * i; c->x_out = xo + i * nd;
      c->F = F_steps ? F_steps + (size_t)(n_cur + (int64_t)i * K) * dim * dim : NULL;
      c->Hlab = F_steps ? HL + 9 * i : NULL;
      c->E = cE + (size_t)i * Kcap; c->tau = cT + (size_t)i * Kcap;
      c->D = cD + (size_t)i * Kcap; c->iters = cI + (size_t)i * Kcap;
    }
    /* level II: P chains (Sec. 3.3, Eq. 19; Algorithm 1 parallel loop) */
    if (n_threads > 1) {
      for (int i0 = 0; i0 < P_eff; i0 += n_threads) {
        int i1 = i0 + n_threads < P_eff ? i0 + n_threads : P_eff;
        for (int i = i0; i < i1; i++) pthread_create(&th[i], NULL, run_chain, &jobs[i]);
        for (int i = i0; i < i1; i++) pthread_join(th[i], NULL);
      }
    } else {
      for (int i = 0; i < P_eff; i++) run_chain(&jobs[i]);
    }
    for (int i = 0; i < P_eff; i++) {
      fire_total += jobs[i].iters_total;
      if (jobs[i].status != ORC_OK) status = jobs[i].status;
    }
    if (status != ORC_OK) break;
    if (wrap_ends)
      for (int i = 0; i < P_eff; i++) orc_wrap(dim, n, xs + (size_t)i * nd, Hs + 9 * i);
    /* sequential equality check (Sec. 3.4, Eq. 20): incoming r_iK | r^c_(i-1)K
     * is the end of chain i-1, outgoing r_iK | r^c_iK is F(r^c_iK); both sit
     * at the strain i dgamma^c, so the minimum image uses chain i's level-I
     * cell (chain i's own cell has moved on by K_i fine steps) */
    int32_t first_fail = -1;
    for (int i = 1; i < P_eff; i++) {
      double m = orc_max_rel_disp(dim, n, xs + (size_t)(i - 1) * nd, xo + (size_t)i * nd, H1 + 9 * i);
      eq[i] = m < eq_tol;
      if (n_log < log_cap) {
        if (log_iter) log_iter[n_log] = iter;
        if (log_i) log_i[n_log] = i;
        if (log_eq) log_eq[n_log] = eq[i];
        if (log_m) log_m[n_log] = m;
      }
      n_log++;
      if (!eq[i]) break;
    }
    int64_t q = orc_alg1_decide(P_eff, Ki, eq, &first_fail);
    /* accepted steps: chains 0..last accepted, in order */
    int last = first_fail < 0 ? P_eff - 1 : first_fail - 1;
    int64_t k = n_cur;
    for (int i = 0; i <= last; i++)
      for (int s = 0; s < Ki[i]; s++, k++) {
        if (E_k) E_k[k] = cE[(size_t)i * Kcap + s];
        if (tau_k) tau_k[k] = cT[(size_t)i * Kcap + s];
        if (iters_k) iters_k[k] = cI[(size_t)i * Kcap + s];
        if (D_k) D_k[k] = cD[(size_t)i * Kcap + s];
      }
    /* r_star <- r_q (end of chain `last`), H follows */
    memcpy(x, xs + (size_t)last * nd, nd * sizeof(double));
    memcpy(H, Hs + 9 * last, sizeof(double) * dim * dim);
    if (F_steps) memcpy(Hlab, HL + 9 * last, sizeof(double) * dim * dim);
    n_cur += q;
    iter++;
    if (adaptive) {
      /* dynamic K: longer chains after a clean pass, after a failed test
       * chains that together span the distance this pass advanced */
      if (first_fail < 0) K = 2 * K < Kcap ? 2 * K : Kcap;
      else K = (int)((q + P - 1) / P) > 1 ? (int)((q + P - 1) / P) : 1;
    }
  }
  if (stats) {
    stats->iterations = iter;
    stats->fire_iters_total = fire_total;
    stats->n_log = n_log;
  }
  free(xs); free(xo); free(Hs); free(H1); free(HL); free(cE); free(cT); free(cD); free(cI);
  free(jobs); free(th); free(Ki); free(eq);
  return status;
}
