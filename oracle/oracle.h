/*
 * oracle.h -- plain FP64 CPU oracle for athermal quasistatic (AQS) deformation
 * stepping and its two-level parallel scheme (Reihn, Bamer, Stamm,
 * "Parallel athermal quasistatic deformation stepping of molecular systems").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and shares no code with it.
 *
 * Everything is FP64, O(N^2) all-pairs, single pass over plain arrays.
 * Conventions (shared with the library by specification, not by code):
 *   - dim d in {2,3}; positions are N x d, row-major, Cartesian.
 *   - the cell is H (d x d, row-major), upper triangular; its columns are the
 *     Bravais vectors (Sec. 2.1).  Simple shear only tilts H[0][1] (Eq. 16).
 *   - minimum image: subtract lattice vectors from the last axis to the
 *     first (z, then y, then x), each by rounding the fractional coordinate
 *     of that axis (reading of the periodic boundaries of Sec. 2.1 for a
 *     sheared cell; valid while the cutoff is below half of every
 *     perpendicular cell width).
 *
 * Readings where the paper is silent are stated next to each function.
 * Functions whose result has no independent pin say "parity unpinned".
 */
#ifndef AQS_ORACLE_H
#define AQS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_TYPES 4

/* status codes (same numbering as the library's, fixed by specification) */
enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = 1,
  ORC_ERR_NOT_CONVERGED = 4,
  ORC_ERR_NONFINITE = 5,
  ORC_ERR_BOX_TOO_SMALL = 7
};

/* Binary Lennard-Jones model (Sec. 2.2, Eq. 13) with a shifted-force cutoff
 * rc_ab = rc_factor * sigma_ab.  sigma/eps are n_types x n_types row-major and
 * symmetric. */
typedef struct {
  int dim;
  int n_types;
  double sigma[ORC_MAX_TYPES * ORC_MAX_TYPES];
  double eps[ORC_MAX_TYPES * ORC_MAX_TYPES];
  double rc_factor;
} orc_potential;

/* FIRE parameters.  The paper minimises with conjugate gradients (Sec. 2.1);
 * the accelerated path uses FIRE, written out in orc_fire(). */
typedef struct {
  double dt0, alpha0, f_inc, f_dec, f_alpha, dt_max, dt_min, max_step, tol;
  int n_min;
  int64_t max_iter;
} orc_fire_params;

/* ---- geometry (Sec. 2.1) ---- */
double orc_volume(int dim, const double* H);
/* in-place minimum image of a separation vector d (length dim) */
void orc_min_image(int dim, const double* H, double* d);
/* largest cutoff allowed by the minimum-image rule: half the smallest
 * perpendicular width of the cell */
double orc_half_min_width(int dim, const double* H);
/* simple-shear affine map F^(dgamma) (Eq. 16): r_i <- F r_i for all atoms
 * (Eq. 3) and H <- F H (Eq. 1) */
void orc_affine_shear(int dim, int n, double* x, double* H, double dgamma);
/* rotates the cell and the configuration rigidly to the frame in which H is
 * upper triangular with a positive diagonal (H = Q R, H <- R, r <- Q^T r);
 * requires det H > 0 */
void orc_triangularise(int dim, int n, double* x, double* H);
/* one deformation increment with a general d x d matrix F (row-major) that
 * acts on the laboratory cell Hlab (in/out, general): Hlab <- F Hlab (Eq. 1).
 * The stored cell H (in/out) is the upper-triangular form of Hlab (Gram-
 * Schmidt frame Q, H = Q^T Hlab) and stored positions follow by
 * M = Q_new^T F Q_old (Eq. 3 in the two frames).  Simple shear (Eq. 16) with
 * Hlab = H gives exactly orc_affine_shear; the paper's pull-push ("pure")
 * shear matrix [[1, dg_x], [dg_y, 1]] (Sec. 2.2) rotates the frame. */
void orc_deform(int dim, int n, double* x, double* H, double* Hlab, const double* F);
/* maps every atom into the cell, r <- r - H floor(H^-1 r) (by whole lattice
 * vectors; the configuration is unchanged under periodic boundaries) */
void orc_wrap(int dim, int n, double* x, const double* H);
/* general affine map with a d x d matrix F (row-major): r_i <- F r_i, H <- F H */
void orc_affine_map(int dim, int n, double* x, double* H, const double* F);

/* ---- energy model (Sec. 2.1 Eqs. 4-6, Sec. 2.2 Eq. 13) ---- */
/* shifted-force LJ pair: for squared distance s returns U_sf(r) and U_sf'(r)
 * (derivative w.r.t. r); zero beyond rc */
void orc_pair_sflj(double s, double sigma, double eps, double rc, double* u, double* du);
/* all-pairs energy E = sum_{i<j} U_sf(r_ij), forces F = -grad E (N x d,
 * nullable) and shear stress tau = (1/V) dE/dgamma (nullable) */
int orc_energy_forces(const orc_potential* pot, int n, const double* x, const int32_t* types,
                      const double* H, double* E, double* F, double* tau);
double orc_fmax(int dim, int n, const double* F);

/* ---- minimiser F of Eq. 10 ---- */
/* FIRE from x (in/out).  Optional traces (length trace_cap, nullable): energy
 * at every force evaluation and a flag that is 1 where the velocity was reset.
 * Returns status; *iters = number of position updates made. */
int orc_fire(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
             const int32_t* types, const double* H, int64_t* iters, double* E, double* fmax,
             double* e_trace, uint8_t* reset_trace, int64_t trace_cap);
/* Polak-Ribiere conjugate gradients with Armijo backtracking (monotone by
 * construction); the paper's own choice of minimiser (Sec. 2.1). */
int orc_cg(const orc_potential* pot, int n, double* x, const int32_t* types, const double* H,
           double tol, int64_t max_iter, int64_t* iters, double* E, double* fmax,
           double* e_trace, int64_t trace_cap);

/* ---- equality and non-affine displacement ---- */
/* max over atoms of | mi(a_i - b_i) - mean_j mi(a_j - b_j) |  (both at the
 * same H); used for the basin test (Eq. 20) and the per-step non-affine
 * displacement D_k */
double orc_max_rel_disp(int dim, int n, const double* a, const double* b, const double* H);

/* ---- AQS protocol (Eq. 12) ---- */
/* n_steps sequential steps of r <- F(F_N^(dgamma) r).  x, H in/out.  Per-step
 * outputs (length n_steps, each nullable): energy E_k, stress tau_k, FIRE
 * iterations, non-affine displacement D_k. */
int orc_aqs(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
            const int32_t* types, double* H, double dgamma, int n_steps, double* E_k,
            double* tau_k, int64_t* iters_k, double* D_k);
/* the same protocol under a deformation history: step k applies the k-th
 * d x d matrix of F (n_steps x d x d, row-major) to the laboratory cell Hlab
 * (in/out; must be given with F) by orc_deform instead of the simple shear
 * by dgamma (F = NULL gives orc_aqs).  Covers pure (pull-push) shear
 * (Sec. 2.2) and cyclic protocols (Sec. 5). */
int orc_aqs_history(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
                    const int32_t* types, double* H, double* Hlab, double dgamma, const double* F,
                    int n_steps, double* E_k, double* tau_k, int64_t* iters_k, double* D_k);

/* ---- two-level parallel stepping (Sec. 3, Algorithm 1) ---- */
typedef struct {
  int64_t iterations;       /* passes of the while loop */
  int64_t fire_iters_total; /* FIRE iterations of all chains, rejected ones included */
  int64_t n_log;            /* entries written to the decision log */
} orc_parallel_stats;

/* Runs Algorithm 1 from the minimum x (in/out, becomes r_{N_steps}).
 * Per accepted step k (length n_steps, nullable): E_k, tau_k, iters_k, D_k.
 * Decision log (capacity log_cap, nullable): for every equality test made,
 * log_iter = while-loop pass, log_i = chain index i, log_eq = 1 if equal,
 * log_m = measured max displacement.  n_threads > 1 runs the level-II
 * chains on that many POSIX threads (the paper's design). */
/* Dynamic K (the paper names an adaptive step count as future work, Sec. 5;
 * this rule is a reading): with K_max > K, the chain length of the next pass
 * is min(K_max, 2 K) after a pass without a failed test and
 * max(1, ceil(q / P)) after a failed test, q the steps that pass accepted.
 * K_max <= K keeps K fixed.  K_pass (nullable, capacity n_steps) receives the
 * K of every pass.  Any K schedule reproduces sequential AQS (Algorithm 1 is
 * exact), which the tests use as the pin.
 * wrap_ends = 1 maps every chain's end into its cell (orc_wrap) before the
 * equality tests.  Positions are only defined up to lattice vectors, so the
 * decisions and the trajectory must not change; the tests use it to check
 * that the tests are made at the shared strain's cell.
 * F_steps (nullable, n_steps x d x d): a deformation history as in
 * orc_aqs_history, with the laboratory cell Hlab in/out; level I then applies
 * the fine increments one after the other (for simple shear F^(a) F^(b) = F^(a+b), so this is the paper's
 * coarse map; for other histories it is the reading that keeps chain i's
 * start in the cell where chain i-1 ends). */
int orc_parallel(const orc_potential* pot, const orc_fire_params* fp, int n, double* x,
                 const int32_t* types, double* H, double dgamma, int K, int P, int n_steps,
                 double eq_tol, int n_threads, double* E_k, double* tau_k, int64_t* iters_k,
                 double* D_k, int64_t* log_iter, int32_t* log_i, uint8_t* log_eq, double* log_m,
                 int64_t log_cap, orc_parallel_stats* stats, int K_max, int32_t* K_pass,
                 int wrap_ends, const double* F_steps, double* Hlab);

/* Pure decision rule of Algorithm 1 (lines after the level-II loop): given
 * the chain lengths K_i (i = 0..P_eff-1) and the equality outcomes eq[i] for
 * i = 1..P_eff-1, returns q (accepted fine steps) and *first_fail (-1 if none). */
int64_t orc_alg1_decide(int P_eff, const int32_t* K_i, const uint8_t* eq, int32_t* first_fail);

/* ---- learned warm start: per-atom features and FP64 MLP ---- */
/* Features of atom i: min-image displacements to its n_nb nearest atoms
 * (ascending distance, ties by index), followed by a one-hot species code of
 * width n_types.  Output n x (n_nb*dim + n_types), row-major. */
int orc_knn_features(int dim, int n, const double* x, const int32_t* types, const double* H,
                     int n_types, int n_nb, double* feat);
/* MLP with GELU hidden layers: layer l maps width[l] -> width[l+1];
 * weights W_l are width[l+1] x width[l] row-major, biases b_l.
 * Forward on m rows of X (m x width[0]); Y is m x width[L]. */
int orc_mlp_forward(int n_layers, const int32_t* width, const double* const* W,
                    const double* const* b, int64_t m, const double* X, double* Y);
/* Mean-squared-error loss 0.5/m * sum (Y - T)^2 and its gradients w.r.t. all
 * weights and biases (dW, db laid out like W, b). */
double orc_mlp_loss_grad(int n_layers, const int32_t* width, const double* const* W,
                         const double* const* b, int64_t m, const double* X, const double* T,
                         double* const* dW, double* const* db);

#ifdef __cplusplus
}
#endif
#endif
