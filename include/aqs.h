/*
 * aqs.h -- C ABI of the GB300 (sm_103a) library for athermal quasistatic (AQS)
 * deformation stepping and its two-level parallel scheme
 * (Reihn, Bamer, Stamm, "Parallel athermal quasistatic deformation stepping
 * of molecular systems").
 *
 * The library holds one or more "replicas" (independent particle systems of
 * the same dimension and potential) on one GPU and runs, per replica:
 *   - the affine deformation F^(dgamma) of the cell and of every atom
 *     (Sec. 2.1, Eqs. 1-3; simple shear, Eq. 16);
 *   - the minimisation operator F: r -> r_inf (Sec. 2.1, Eq. 10), here FIRE
 *     with shifted-force Lennard-Jones forces (Sec. 2.2, Eq. 13) from cell
 *     and Verlet lists under Lees-Edwards periodic boundaries;
 *   - sequential AQS (Eq. 12) and the two-level parallel stepping of Sec. 3
 *     (Algorithm 1) with the equality test of Eq. 20.
 *
 * Conventions
 *   - dim d in {2, 3}.  Positions are N x d row-major Cartesian, in the
 *     caller's atom order ("user order"); the library reorders atoms
 *     internally and always converts back.
 *   - The cell H is d x d row-major, upper triangular; its columns are the
 *     Bravais vectors.  Simple shear adds dgamma * H[1][1] to H[0][1] and
 *     dgamma * y to every x.  The tilt must stay within the minimum-image
 *     rule: cutoff + skin below half of every perpendicular cell width.
 *   - Positions returned by the library may differ from the ones passed in
 *     by whole lattice vectors (atoms are wrapped into the cell when the
 *     neighbour lists are rebuilt); compare configurations by minimum image.
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes; device pointers must be on the library's GPU.
 *
 * Errors: every call returns an aqs_status; no call aborts or throws.  The
 * thread-local text of the last error is available from aqs_last_error().
 * Device code never traps: kernels write a status word that the host reads.
 *
 * Threading: one system is used from one host thread at a time; all work of
 * a system is ordered on the stream given at creation.
 */
#ifndef AQS_H
#define AQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AQS_MAX_TYPES 4

typedef enum {
  AQS_OK = 0,
  AQS_ERR_INVALID_ARG = 1,
  AQS_ERR_CUDA = 2,
  AQS_ERR_OOM = 3,
  AQS_ERR_NOT_CONVERGED = 4,  /* FIRE hit max_iter */
  AQS_ERR_NONFINITE = 5,      /* NaN/Inf force or energy */
  AQS_ERR_NLIST_OVERFLOW = 6, /* internal; the library grows the list and retries */
  AQS_ERR_BOX_TOO_SMALL = 7,  /* cutoff + skin >= half a perpendicular cell width */
  AQS_ERR_TIMEOUT = 8,
  AQS_ERR_UNSUPPORTED = 9
} aqs_status;

typedef enum {
  AQS_FP64 = 0,  /* every force evaluation in FP64 */
  AQS_MIXED = 1  /* FP32 pair forces relative to an FP64 reference force; FP64
                    positions, reductions and final convergence test */
} aqs_precision;

/* Binary (up to 4 species) Lennard-Jones model, Sec. 2.2 Eq. 13, with the
 * shifted-force cutoff rc_ab = rc_factor * sigma_ab:
 *   U_sf(r) = U(r) - U(rc) - (r - rc) U'(rc) for r < rc, 0 beyond.
 * sigma, eps: n_types x n_types row-major, symmetric. */
typedef struct {
  int n_types;
  double sigma[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double eps[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double rc_factor;
} aqs_potential;

typedef struct {
  int dim;                 /* 2 or 3 */
  int n_replicas;          /* >= 1 */
  const int64_t* n_atoms;  /* host [n_replicas]; each >= 2 */
  const double* box;       /* host [n_replicas * dim * dim], H per replica */
  const double* pos;       /* host or device [sum n_atoms * dim], user order */
  const int32_t* types;    /* host or device [sum n_atoms], values < n_types */
  aqs_potential pot;
  aqs_precision precision;
  double skin;             /* Verlet skin; <= 0 selects 0.3 */
  int nlist_capacity;      /* neighbours per atom; <= 0 selects 64 (2D) / 160 (3D) */
  int cluster_size;        /* CTAs per replica (1..16); <= 0 selects automatically */
  void* stream;            /* cudaStream_t for all work; NULL = legacy default stream */
  /* optional device allocator (e.g. a framework's caching allocator); both
   * NULL selects cudaMalloc/cudaFree.  Blocks must be 16-byte aligned (the
   * kernels use 16-byte vector and 8-byte atomic accesses); a misaligned
   * block fails the call with AQS_ERR_OOM.  The library never frees what it
   * did not allocate. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
} aqs_system_desc;

typedef struct aqs_system aqs_system; /* opaque; owns all device state */

/* FIRE controls (the minimiser F of Eq. 10).  The library's FIRE:
 *   P = F.v; P >= 0: npos++, after n_min such steps dt = min(dt*f_inc, dt_max),
 *   alpha *= f_alpha; P < 0: npos = 0, dt = max(dt*f_dec, dt_min),
 *   alpha = alpha0, v = 0; then v += dt F, v = (1-alpha) v + alpha |v|/|F| F,
 *   per-atom step dt v capped at max_step.  Converged when max_a |F_a| < tol
 *   (tested before moving; in AQS_MIXED always on an FP64 evaluation).
 * ref_ratio / ref_dmax (AQS_MIXED only): a new FP64 reference force is taken
 * when an atom has moved more than min(ref_ratio * fmax, ref_dmax) from the
 * reference positions. */
typedef struct {
  double dt0, alpha0, f_inc, f_dec, f_alpha, dt_max, dt_min, max_step, tol;
  int n_min;
  int64_t max_iter;
  double ref_ratio, ref_dmax;
} aqs_fire_params;

/* dt0 0.005, alpha0 0.1, f_inc 1.1, f_dec 0.5, f_alpha 0.99, dt_max 0.05,
 * dt_min 1e-4, max_step 0.1, tol 1e-10, n_min 5, max_iter 1e6,
 * ref_ratio 30, ref_dmax 0.05 */
void aqs_fire_params_default(aqs_fire_params* out);

typedef struct {
  int64_t iters;     /* FIRE position updates */
  int64_t evals64;   /* FP64 force evaluations (every evaluation in AQS_FP64) */
  int64_t rebuilds;  /* neighbour-list rebuilds during the call */
  double energy;     /* U at the minimum (FP64) */
  double fmax;       /* max_a |F_a| at the minimum (FP64) */
  double tau;        /* shear stress (1/V) dU/dgamma at the minimum */
  double nonaffine;  /* max_a |(r_a - r_a^start) - mean| over the call */
  int status;        /* aqs_status of this replica */
} aqs_min_result;

/* Creates a system; copies pos/types.  Fails with AQS_ERR_BOX_TOO_SMALL when
 * the cell is too small for the cutoff and skin, and with AQS_ERR_NONFINITE
 * when a position is NaN or infinite. */
aqs_status aqs_create_system(const aqs_system_desc* desc, aqs_system** out);
void aqs_destroy_system(aqs_system* sys);

/* Simple shear F^(dgamma) (Eq. 16) of every atom and of the cell of each
 * replica; dgamma: host [n_replicas] (a replica with 0 is untouched). */
aqs_status aqs_affine_shear(aqs_system* sys, const double* dgamma);

/* Minimisation operator F (Eq. 10) on all replicas with mask[r] != 0
 * (mask NULL = all), batched in one persistent launch per pass.
 * out: host [n_replicas] (entries of masked-out replicas untouched);
 * returns the first non-OK replica status, else AQS_OK. */
aqs_status aqs_minimize(aqs_system* sys, const aqs_fire_params* fire, const uint8_t* mask,
                        aqs_min_result* out);

/* Sequential AQS (Eq. 12) on every replica at once: n_steps times
 * [affine dgamma; minimise].  Per-step outputs, host, [n_steps * n_replicas]
 * step-major (nullable each): energy, tau, FIRE iterations, non-affine
 * displacement D_k = max_a |mi(r_k,a - (F r_{k-1})_a) - mean|. */
aqs_status aqs_run_sequential(aqs_system* sys, const aqs_fire_params* fire, double dgamma,
                              int64_t n_steps, double* energy, double* tau, int64_t* fire_iters,
                              double* nonaffine);

/* Two-level parallel stepping, Algorithm 1 (Sec. 3.5), from the minimum held
 * in `replica` (r_star).  Level I makes P affine predictions
 * F^(i K dgamma) r_star (Eq. 18); level II runs the P chains
 * (F o F_N)^K o F (Eq. 19) as replicas of one batched launch; the equality
 * test (Eq. 20) compares, for i = 1..P-1, the end of chain i-1 with F(r^c_iK)
 * by max_a |mi(a - b) - mean| < eq_tol; r_star <- r_q.
 * Readings: the last window runs P_eff = min(P, ceil(rem/K)) chains, the last
 * one shortened to end exactly at n_steps; a step is a plastic event when its
 * D_k exceeds event_threshold. */
typedef struct {
  double dgamma;          /* fine increment */
  int K;                  /* fine steps per chain (>= 1) */
  int P;                  /* chains (>= 1) */
  int64_t n_steps;        /* fine steps to advance in this call */
  double eq_tol;          /* <= 0 selects 1e-6 */
  double event_threshold; /* <= 0 selects 1e-2 */
  int64_t max_iterations; /* while-loop passes in this call; <= 0: until n_steps */
  int warm_start;         /* 1: start each fine minimisation from the learned
                             prediction (see aqs_warm_*); 0: plain affine start */
  int run_discarded;      /* 0 (default): a chain stops as soon as a failed
                             equality test of an earlier or the same chain
                             index shows that its result will be discarded;
                             1: every chain runs to its end as in the paper.
                             Results and decisions are identical. */
  int K_max;              /* dynamic K (the paper leaves an adaptive step count
                             to future work, Sec. 5): with K_max > K the next
                             pass uses min(K_max, 2 K) after a pass without a
                             failed test and max(1, ceil(q / P)) after one, q the
                             steps that pass accepted; <= K keeps K fixed.  The
                             trajectory is that of sequential AQS either way. */
  const double* F_steps;  /* nullable: a deformation history for this call,
                             host [n_steps][dim][dim] (see aqs_run_history);
                             fine step k applies F_steps[k] instead of the
                             simple shear by dgamma, and level I maps chain i
                             by the i K increments that follow the current
                             step, one after the other (for simple shear this
                             is the paper's F^(i K dgamma); for a general
                             history it keeps chain i's start in the cell where
                             chain i-1 ends).  Not with warm_start. */
} aqs_parallel_params;

typedef struct {
  int64_t iterations;       /* while-loop passes made */
  int64_t accepted_steps;   /* fine steps accepted (= advance of r_star) */
  int64_t rejections;       /* passes that ended at a failed equality test */
  int64_t fire_iters_total; /* FIRE iterations of all chains, rejected ones included */
  int64_t evals64_total;    /* FP64 force evaluations of all chains */
  int64_t chains_stopped;   /* chains stopped early (see run_discarded) */
  int32_t* K_pass;          /* nullable, capacity n_steps: K of every pass */
  int32_t K_next;           /* K the next pass would use (dynamic K; pass it as
                               K to continue pass by pass) */
  /* caller-allocated host arrays indexed by accepted step (nullable each),
   * capacity n_steps: */
  double* energy;
  double* tau;
  int64_t* fire_iters;
  double* nonaffine;
  uint8_t* event;
  /* decision log, caller-allocated, capacity log_cap: one entry per equality
   * test made (pass, chain index i, equal?, measured displacement) */
  int64_t log_cap;
  int64_t n_log;
  int64_t* log_iter;
  int32_t* log_i;
  uint8_t* log_eq;
  double* log_m;
} aqs_parallel_result;

aqs_status aqs_parallel_step(aqs_system* sys, int replica, const aqs_fire_params* fire,
                             const aqs_parallel_params* params, aqs_parallel_result* out);

/* ---- general deformation histories ----
 * The paper's protocol uses simple shear (Eq. 16) and states that the method
 * works as well for pull-push ("pure") shear F = [[1, dg_x], [dg_y, 1]]
 * (Sec. 2.2) and for other deformation histories such as cyclic protocols
 * (Sec. 5).  An increment F (d x d, row-major) acts on the laboratory cell:
 * H_lab <- F H_lab, r <- F r (Eqs. 1-3).  The library keeps every cell upper
 * triangular: it stores H = Q^T H_lab with Q the Gram-Schmidt frame of H_lab
 * (aqs_get_frame) and the configuration in that frame, so stored positions
 * move by the upper-triangular map Q_new^T F Q_old.  For simple shear Q stays
 * the identity.  3D histories must keep the stored cell tilted in xy only
 * (AQS_ERR_UNSUPPORTED otherwise); every cell reached must satisfy the
 * minimum-image rule (AQS_ERR_BOX_TOO_SMALL, nothing applied). */

/* One increment per replica: F host [n_replicas][dim][dim].  Lists are
 * rebuilt in the new cell. */
aqs_status aqs_deform(aqs_system* sys, const double* F);
/* Sequential AQS (Eq. 12) under a deformation history: step k applies
 * F[k] (host [n_steps][dim][dim], the same history for every replica), then
 * minimises.  Outputs as aqs_run_sequential. */
aqs_status aqs_run_history(aqs_system* sys, const aqs_fire_params* fire, const double* F,
                           int64_t n_steps, double* energy, double* tau, int64_t* fire_iters,
                           double* nonaffine);
/* Q (host [dim][dim], row-major): laboratory = Q x stored, for positions and
 * cell; the identity unless a history rotated the cell. */
aqs_status aqs_get_frame(const aqs_system* sys, int replica, double* Q);

/* Equality test of Eq. 20 between replica ra of a and replica rb of b (same
 * atom count, same cell): max_disp = max_a |mi(r_a - r_b) - mean|,
 * equal = max_disp < tol.  The two systems must share one stream. */
aqs_status aqs_compare_configs(const aqs_system* a, int ra, const aqs_system* b, int rb,
                               double tol, double* max_disp, int* equal);

/* ---- state access ---- */
int aqs_num_replicas(const aqs_system* sys);
int64_t aqs_num_atoms(const aqs_system* sys, int replica);
/* out: host or device [n * dim], user order */
aqs_status aqs_get_positions(const aqs_system* sys, int replica, double* out);
/* pos: host or device [n * dim], user order; resets FIRE state of the replica;
 * AQS_ERR_NONFINITE (nothing written) if a coordinate is NaN or infinite */
aqs_status aqs_set_positions(aqs_system* sys, int replica, const double* pos);
aqs_status aqs_get_box(const aqs_system* sys, int replica, double* H);
aqs_status aqs_set_box(aqs_system* sys, int replica, const double* H);
/* FP64 energy, forces (host or device [n * dim], user order, nullable) and
 * shear stress (nullable) of one replica at its current positions */
aqs_status aqs_energy_forces(aqs_system* sys, int replica, double* energy, double* forces,
                             double* tau);

/* ---- learned warm start (2D) ----
 * The paper names extrapolation of the minimiser's starting point as future
 * work (Sec. 5).  A per-atom network predicts the non-affine displacement per
 * unit strain u_i of the next increment from the atom's neighbour shell; the
 * minimisation starts from F^(dgamma) r_k + dgamma u and FIRE finishes it.
 *
 * Features of atom i (aqs_warm_features): the minimum-image displacements to
 * its 32 nearest atoms, nearest first (ties: lower caller index first), then a
 * one-hot species code (width 66 in 2D; BF16 rows are padded with zeros to
 * AQS_WARM_IN = 80).  Rows are in caller order; with replica = -1 the rows of
 * replica r start at the sum of the sizes of the replicas before it.
 * Network: 80 -> 128 -> 128 -> 128 -> 2, GELU on the hidden layers, BF16
 * weights and activations on tensor cores, FP32 accumulation, FP32 master
 * weights; loss 0.5/m sum (y - t)^2; AdamW (beta 0.9, 0.999, eps 1e-8).
 * Parameter vector (aqs_warm_num_params floats): W1 (128 x 80), W2, W3
 * (128 x 128), W4 (16 x 128, rows >= 2 zero), b1, b2, b3 (128), b4 (16). */
#define AQS_WARM_IN 80
typedef struct aqs_warm aqs_warm;
int aqs_warm_num_params(void);
/* Glorot-uniform weights from a SplitMix64 stream of `seed`, zero biases. */
aqs_status aqs_warm_create(int dim, int n_types, uint64_t seed, void* stream, aqs_warm** out);
void aqs_warm_destroy(aqs_warm* w);
aqs_status aqs_warm_get_params(const aqs_warm* w, float* host_params);
aqs_status aqs_warm_set_params(aqs_warm* w, const float* host_params); /* resets AdamW state */
/* feat_bf16: device [rows][80]; feat_f64: device [rows][66] or NULL */
aqs_status aqs_warm_features(aqs_system* sys, int replica, void* feat_bf16, double* feat_f64);
/* feat_bf16: device [rows][80], 16-byte aligned (AQS_ERR_INVALID_ARG otherwise);
 * out: device [rows][2] FP32 */
aqs_status aqs_warm_predict(aqs_warm* w, const void* feat_bf16, int64_t rows, float* out);
/* loss and its gradient (host, aqs_warm_num_params floats, nullable) for
 * targets (device [rows][2] FP32) */
aqs_status aqs_warm_loss_grad(aqs_warm* w, const void* feat_bf16, const float* target,
                              int64_t rows, float* grad_host, double* loss);
/* one AdamW step on the full-batch gradient of the given rows */
aqs_status aqs_warm_train_step(aqs_warm* w, const void* feat_bf16, const float* target,
                               int64_t rows, double lr, double weight_decay, double* loss);
/* Training data from the method itself: n_steps sequential AQS steps of all
 * replicas; before each step the features of the current minima, after it
 * the per-atom non-affine displacement per unit strain (targets).
 * feat_out: device [n_steps][N_tot][80] BF16; target_out: device
 * [n_steps][N_tot][2] FP32. */
aqs_status aqs_warm_collect(aqs_system* sys, const aqs_fire_params* fire, double dgamma,
                            int64_t n_steps, void* feat_out, float* target_out);
/* Sequential AQS with the learned start.  A step keeps it only if the
 * minimum lies within `gate` (<= 0 selects 0.01 sigma) of both the learned
 * start and the plain affine start (an elastic step, so both starts lie in one
 * basin); otherwise the step is redone from the plain affine start, which
 * defines the AQS path (Eq. 12).  Per-step outputs as aqs_run_sequential;
 * used_warm[i] = 1 where the learned start was kept; fire_iters includes the
 * iterations of a discarded attempt. */
aqs_status aqs_run_sequential_warm(aqs_system* sys, const aqs_fire_params* fire, aqs_warm* w,
                                   double dgamma, int64_t n_steps, double gate, double* energy,
                                   double* tau, int64_t* fire_iters, double* nonaffine,
                                   uint8_t* used_warm);

/* ---- allocation-free evaluation ----
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate device memory (inside another library's fixed memory
 * plan, under an allocation quota, or while holding a lock that cudaMalloc
 * could wait on).  It computes the FP64 shifted-force LJ energy, forces and
 * shear stress of ONE configuration by visiting all pairs (minimum image),
 * with no system, no Verlet list and no cudaMalloc/cudaFree or other
 * allocating call.  Its only scratch is a fixed device array inside the
 * library (one partial sum pair per 128 atoms, AQS_NOALLOC_MAX_ATOMS atoms at
 * most, 8 KiB held on every GPU that loads the library until the process
 * exits).
 *   dim       2 or 3
 *   n         atoms, 2 <= n <= AQS_NOALLOC_MAX_ATOMS, else AQS_ERR_INVALID_ARG
 *   pos       device [n * dim], Cartesian
 *   types     device [n], values < pot->n_types
 *   box       host [dim * dim], upper-triangular cell with its tilt in H[0][1]
 *             only (any other off-diagonal entry: AQS_ERR_INVALID_ARG);
 *             AQS_ERR_BOX_TOO_SMALL if 2 * max cutoff >= a perpendicular width
 *   pot       host, the potential as in aqs_potential
 *   forces    device [n * dim], written (force on each atom)
 *   energy_tau device [2], written: total energy, shear stress (1/V) dU/dgamma
 *   stream    cudaStream_t (NULL = legacy default stream); the call only
 *             enqueues work and returns without synchronising.
 * Every call looks up the scratch array's device address with
 * cudaGetSymbolAddress in the caller's current context (the address belongs
 * to the context, so it is not cached).  The first call on a device also makes
 * the runtime load the library's device code there; make that first call
 * before capturing a stream.  Every call shares the one scratch array and each
 * call overwrites every slot it later reads, so nothing has to be cleared, but
 * calls that overlap on the GPU (different streams, no ordering) race on it. */
#define AQS_NOALLOC_MAX_ATOMS 65536
aqs_status aqs_energy_forces_noalloc(int dim, int64_t n, const double* pos, const int32_t* types,
                                     const double* box, const aqs_potential* pot, double* forces,
                                     double* energy_tau, void* stream);

/* ---- launch configuration: cluster size, staging mode, autotuner ----
 * The paper runs one chain per CPU thread (Sec. 3.3); here every replica is
 * minimised by one thread-block cluster of C CTAs, and C trades atoms per
 * thread against how many replicas are resident at once.  The staging mode
 * says where a CTA finds its list rows and its neighbours' position records:
 *   0  rows from global memory each iteration, records from global memory
 *   1  rows staged in shared memory, records read from the owner CTA (DSMEM)
 *   2  rows staged, the whole replica's records copied into shared memory
 *   3  rows staged, records from global memory
 * Every mode reads the same values, so results are bitwise identical; only
 * speed and shared-memory needs differ (a mode that does not fit falls back
 * to the automatic choice: 2, else 1, else 0). */

/* Times `iters` FIRE iterations (convergence test disabled, so every candidate
 * does the same work from the same configuration) of the replicas with
 * mask[r] != 0 (NULL = all): every feasible C in 1..16 (at most 4096 and at
 * least 32 atoms per CTA, at least one cluster resident), each with every
 * staging mode that fits and with one and (where it fits) two threads per
 * atom in the force phase, and the same sizes again as one cooperative launch
 * with grid barriers (aqs_set_grid_barrier; staging modes 0 and 3) (the staging mode sets a CTA's shared memory and so
 * how many CTAs of different clusters share an SM, i.e. how many replicas'
 * clusters are resident at once).  Keeps the fastest (C, staging, threads per
 * atom, barrier mode), except what aqs_set_staging / aqs_set_threads_per_atom /
 * aqs_set_grid_barrier fixed;
 * ms_per_iter[C] is the fastest candidate at C.
 * Outputs, each may be NULL: *best_cluster, *best_staging;
 * ms_per_iter[17] (entry C: wall time per iteration in ms, -1 if C was not
 * feasible; entry 0 unused); ms_per_staging[4] (entry m: time per iteration
 * at the best C and threads per atom in mode m, -1 if not timed).  Positions, boxes and minimiser
 * state are restored afterwards, so tuning does not change the
 * configuration.  Errors as aqs_minimize, except that not converging is the
 * expected outcome. */
aqs_status aqs_autotune_clusters(aqs_system* sys, const aqs_fire_params* fire, int64_t iters,
                                 const uint8_t* mask, int* best_cluster, int* best_staging,
                                 double* ms_per_iter, double* ms_per_staging);
/* With iters > 0, every later minimisation (aqs_minimize, aqs_run_sequential,
 * the chains of aqs_parallel_step) first tunes cluster size and staging for
 * its set of replicas in flight, once per (number of replicas, largest N),
 * and reuses the cached choice afterwards.  0 switches it off (the default
 * size rule: C = min(16, 152 / replicas), at least ceil(N / 4096)).  Ignored
 * when the system was created with an explicit cluster_size. */
aqs_status aqs_set_autotune(aqs_system* sys, int64_t iters);
/* FIRE iterations (>= 1, default 2048) each replica runs per persistent
 * launch before control returns to the host, which then gives the replicas
 * still running larger clusters and stops discarded level-II chains.
 * Shorter launches use the GPU better when replicas finish at different
 * times, at the cost of a host round trip and one FP64 force evaluation per
 * replica per launch.  Results agree within the precision's tolerance (the
 * FP64 re-reference points move).  Applies to the system and its chains. */
aqs_status aqs_set_launch_budget(aqs_system* sys, int64_t iters);
/* Threads per atom in the force phase of the minimiser ("atoms per warp"
 * 32 / tpa): 1, or 2 (each atom's list split between two adjacent lanes that
 * sum their partial forces in a fixed order; used where 2 x atoms-per-CTA
 * threads fit a CTA, else 1), or 0 to let the autotuner choose (1 without
 * it).  Applies to the system and its chains.  Results agree with tpa = 1
 * within rounding (the force sums are added in another order). */
aqs_status aqs_set_threads_per_atom(aqs_system* sys, int tpa);
int aqs_threads_per_atom(const aqs_system* sys);
/* on = 1: the minimiser runs the replicas' CTAs in one cooperative launch
 * without thread-block clusters; the CTAs of a replica synchronise through a
 * barrier in global memory (bounded waits: a wait that runs out ends the
 * call with AQS_ERR_TIMEOUT) and read neighbour records from global memory
 * (staging modes 0 and 3).  The device holds clusters per GPC, which limits
 * how many replicas fit at a given cluster size (e.g. 15 clusters of 7-9 CTAs
 * on a GB300); a cooperative launch is limited only by resident CTAs.  One
 * cluster size for all replicas of a launch.  on = 0: thread-block clusters;
 * on = -1 (the default): the autotuner (aqs_set_autotune) times both and keeps
 * the faster, clusters without it.  Applies to the system and its chains.
 * Results agree within rounding with the cluster launches. */
aqs_status aqs_set_grid_barrier(aqs_system* sys, int on);
/* The barrier mode the minimiser launches use: of this system (of_chains =
 * 0) or of its level-II chains (of_chains = 1): 1 grid barriers, 0 clusters
 * (after autotuning, the mode it kept); -1 if the chains have not run yet or
 * sys is NULL. */
int aqs_grid_barrier(const aqs_system* sys, int of_chains);
/* How many clusters of C CTAs of this replica's minimiser launch the device
 * can hold at once (cudaOccupancyMaxActiveClusters) for a staging mode
 * (-1 automatic) and threads per atom; -1 on a bad argument. */
int aqs_max_active_clusters(const aqs_system* sys, int replica, int C, int staging, int tpa);
/* Fixes the staging mode (0..3) of this system and its chains, or -1 for the
 * automatic choice.  AQS_ERR_INVALID_ARG outside -1..3. */
aqs_status aqs_set_staging(aqs_system* sys, int mode);
/* Staging mode a launch of this replica alone would use (-1 on a bad argument). */
int aqs_staging(const aqs_system* sys, int replica);

/* ---- diagnostics ---- */
/* Counters of the persistent minimiser kernel, accumulated over all systems
 * while timing is on (aqs_set_kernel_timing(1)); pair visits count one atom
 * looking at one list entry (a pair is visited from both sides). */
typedef struct {
  int64_t launches;      /* minimiser launches */
  double kernel_ms;      /* sum of their durations (CUDA events on the system stream) */
  int64_t evals32;       /* FP32 relative force evaluations (all replicas) */
  int64_t evals64;       /* FP64 force evaluations (all replicas) */
  int64_t pairs32;       /* pair visits in FP32 evaluations */
  int64_t pairs64;       /* pair visits in FP64 evaluations */
  int64_t atom_iters;    /* atoms x FIRE iterations */
  int64_t rebuilds;      /* Verlet-list rebuilds done inside the minimiser kernel */
} aqs_kernel_stats;
void aqs_set_kernel_timing(int on);
void aqs_get_kernel_stats(aqs_kernel_stats* out);
void aqs_reset_kernel_stats(void);

const char* aqs_last_error(void);
/* number of kernels this library launched in this process */
int64_t aqs_launch_count(void);
/* mean neighbour-list length of a replica after the last rebuild */
double aqs_mean_neighbours(const aqs_system* sys, int replica);
int aqs_cluster_size(const aqs_system* sys, int replica);

#ifdef __cplusplus
}
#endif
#endif /* AQS_H */
