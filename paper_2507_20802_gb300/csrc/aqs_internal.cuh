// aqs_internal.cuh -- device-side data layout and shared helpers of the AQS
// library (sm_103a).  Not part of the public ABI.
//
// Layout in HBM (one system = R replicas of N_r atoms each, N_tot atoms):
//   per-atom FP64 arrays are structure-of-arrays, component-major:
//     x[c * N_tot + i]  (c < dim), atoms of replica r at [off_r, off_r + N_r)
//     in cell-sorted order; perm[i] gives the caller's index within the replica.
//   Verlet list of replica r: column-major block nb[nb_off_r + k * N_r + i],
//     k < cap, one 32-bit entry per neighbour (see encode_nb below).
//   Per-replica geometry (RepGeom, written by the host) and minimiser state
//   (RepState, written by the kernels) live in small device arrays.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aqs.h"

namespace aqs {

constexpr int kMaxTypes = AQS_MAX_TYPES;
constexpr int kMaxCluster = 16;
constexpr int kNumRed = 8;  // reduction slots per iteration

// Shifted-force LJ pair coefficients for one type pair (a, b).  With
// d = r_j - r_i and s = |d|^2 the force on atom i is phi(s) d with
//   phi(s) = U_sf'(r) / r = A s^-7 + B s^-4 + C s^-1/2,
//   A = -48 eps sig^12, B = 24 eps sig^6, C = -U'(rc)       (Sec. 2.2, Eq. 13)
// and the energy U_sf(r) = e12 s^-6 - e6 s^-3 - Uc - (r - rc) dUc.
struct PairCoef {
  double A, B, C;
  double rc2, rl2;  // cutoff^2 and (cutoff + skin)^2
  double e12, e6, Uc, dUc, rc;
  float Af, Bf, Cf, rc2f;
};

struct RepGeom {
  int64_t off;     // first atom (global index)
  int64_t nb_off;  // first list entry
  int n;           // atoms
  int C;           // CTAs (cluster size) that own this replica
  int npc;         // atoms per CTA = ceil(n / C)
  int cell_off;    // first cell (global cell index)
  int nc[3];       // cells per axis (fractional-coordinate grid)
  int ncell;       // nc[0] * nc[1] * nc[2]
  double H[9];     // current cell, row-major dim x dim (upper triangular)
  double tilt_b;   // H[0][1] when the list was built
};

// Minimiser state of one replica, written by the kernel.  A replica runs a
// "job" of nsteps fine steps (affine dgamma, then FIRE to convergence); the
// first step skips the affine map when first_noaffine is set (the level-II
// chains' first minimisation).  A launch may stop inside a job (list rebuild,
// iteration budget) and the next launch resumes it.
struct RepState {
  double dt, alpha;
  double E, fmax, tau;
  double tilt;      // current H[0][1] (authoritative; the host mirrors it)
  double tilt_b;    // H[0][1] when the list was built (host-written)
  double dgamma;    // fine increment of the job
  int64_t iters;    // FIRE position updates of the current step
  int64_t evals64;  // FP64 force evaluations of the current step
  int64_t evals32;  // FP32 (relative) force evaluations of the current step
  int64_t acc_iters, acc64, acc32;  // monotonic counters over all launches
  int64_t step;     // steps of the job completed
  int64_t nsteps;   // steps of the job
  int npos;
  int status;       // aqs_status; kStatusRebuild / kStatusRunning while unfinished
  int phase;        // 0: next step not started, 1: FIRE in progress
  int first_noaffine;
  int want_snap;    // write the positions after the first (no-affine) step
  int kreb;         // Verlet rebuilds done inside the kernel (monotonic)
  // Deformation histories (launches with a map table): the current cell,
  // authoritative while such a job runs, and the cell at the last list build.
  double Hc[9];
  double Hb[9];
};

// Deformation-history table: per replica and job step, the map M of stored
// positions (upper triangular, row-major 3 x 3 slots) and the new stored cell.
constexpr int kHistFields = 18;

// per converged step the kernel records: E, tau, D_k (from the affine start), FIRE
// iterations, FP64 evaluations, max displacement from the minimisation's start
constexpr int kRecFields = 6;

constexpr int kStatusRebuild = 100;
constexpr int kStatusRunning = 101;

struct FireDev {
  double dt0, alpha0, f_inc, f_dec, f_alpha, dt_max, dt_min, max_step, tol;
  double ref_ratio, ref_dmax;
  int n_min;
  int64_t max_iter;
};

// Neighbour entry: slot (14 bits) within the owner CTA, owner CTA rank
// (4 bits), neighbour-cell offset code (5 bits: (a+1) + 3 (b+1) + 9 (c+1)),
// neighbour species (2 bits).
__host__ __device__ inline uint32_t encode_nb(int slot, int owner, int code, int type) {
  return (uint32_t)slot | ((uint32_t)owner << 14) | ((uint32_t)code << 18) | ((uint32_t)type << 23);
}
__device__ inline int nb_slot(uint32_t e) { return (int)(e & 0x3FFFu); }
__device__ inline int nb_owner(uint32_t e) { return (int)((e >> 14) & 0xFu); }
__device__ inline int nb_code(uint32_t e) { return (int)((e >> 18) & 0x1Fu); }
__device__ inline int nb_type(uint32_t e) { return (int)((e >> 23) & 0x3u); }
constexpr int kMaxSlot = 1 << 14;

// Cartesian offset between the origins of two cells that are (a, b, c)
// cells apart on the fractional grid: H (a/nx, b/ny, c/nz).  Wrapping a cell
// index across the periodic boundary and adding the lattice image cancel, so
// d_ij = q_j - q_i + offset(code) with q the position relative to the atom's
// own cell origin.
template <int D>
__host__ __device__ inline void cell_offset(const double* H, const int* nc, int code, double* o) {
  int a = code % 3 - 1, b = (code / 3) % 3 - 1, c = code / 9 - 1;
  double f[3] = {(double)a / nc[0], (double)b / nc[1], D == 3 ? (double)c / nc[2] : 0.0};
  for (int r = 0; r < D; r++) {
    double s = 0.0;
    for (int k = r; k < D; k++) s += H[r * D + k] * f[k];
    o[r] = s;
  }
}

template <int D>
__host__ __device__ inline void cell_origin(const double* H, const int* nc, int cell, double* o) {
  int cx = cell % nc[0], cy = (cell / nc[0]) % nc[1], cz = D == 3 ? cell / (nc[0] * nc[1]) : 0;
  double f[3] = {(double)cx / nc[0], (double)cy / nc[1], D == 3 ? (double)cz / nc[2] : 0.0};
  for (int r = 0; r < D; r++) {
    double s = 0.0;
    for (int k = r; k < D; k++) s += H[r * D + k] * f[k];
    o[r] = s;
  }
}

// Frobenius norm of H Hb^-1 - I for upper-triangular cells: the largest
// relative change (bound) of any separation vector under the affine maps
// applied since the cell was Hb.  For simple shear it is |dt| / L_y.
template <int D>
__host__ __device__ inline double affine_change(const double* H, const double* Hb) {
  double A[9];
  // A Hb = H, column by column (Hb upper triangular)
  for (int c = 0; c < D; c++)
    for (int r = 0; r < D; r++) {
      double v = H[r * D + c];
      for (int k = 0; k < c; k++) v -= A[r * D + k] * Hb[k * D + c];
      A[r * D + c] = v / Hb[c * D + c];
    }
  double f = 0.0;
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) {
      const double e = A[r * D + c] - (r == c ? 1.0 : 0.0);
      f += e * e;
    }
  return sqrt(f);
}

// Minimum image of a separation d under the upper-triangular cell H: remove
// lattice vectors from the last axis to the first, rounding the fractional
// coordinate of each axis.
template <int D>
__device__ inline void min_image(const double* H, double* d) {
#pragma unroll
  for (int c = D - 1; c >= 0; c--) {
    double n = rint(d[c] / H[c * D + c]);
#pragma unroll
    for (int a = 0; a <= c; a++) d[a] -= n * H[a * D + c];
  }
}

}  // namespace aqs
