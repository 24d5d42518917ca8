// minimize.cu -- persistent FIRE minimiser, one thread-block cluster per
// replica (the minimisation operator F of Sec. 2.1, Eq. 10).
//
// Each replica is owned by a cluster of C CTAs (C <= 16); CTA `rank` owns the
// atoms [rank * npc, (rank + 1) * npc) of the replica's cell-sorted order and
// publishes their positions in its shared memory (and, in staging modes 0 and
// 3, in a global record array).  Neighbour positions are read from the owner
// CTA through distributed shared memory (DSMEM), from a shared-memory copy of
// the whole replica, or from the global records (the staging modes listed in
// minimize.cuh).  One FIRE
// iteration is:
//   force phase   -- pair forces of the owned atoms from the Verlet list,
//                    per-thread partial sums of the FIRE reductions;
//   reduction     -- warp shuffles, CTA tree, cluster barrier, every CTA sums
//                    the C partials in rank order (bitwise identical totals in
//                    all CTAs, so every control decision is uniform);
//   update phase  -- FIRE velocity/position update of the owned atoms and
//                    publication of the new positions; cluster barrier.
// The loop runs until convergence, the iteration cap, a non-finite force or a
// tripped Verlet skin (then the replica waits for a list rebuild and the next
// launch resumes the same FIRE state).
//
// Precision modes (aqs_precision):
//   AQS_FP64  -- every force evaluation in FP64 ("EVAL64").
//   AQS_MIXED -- positions are x = x_ref + delta with an FP64 reference force
//                F_ref = F(x_ref).  Between references the force is
//                F_ref + dF, where dF = sum_j [phi(s) d - phi(s0) d0] is
//                computed in FP32 from the reference separation d0 and the
//                small relative displacement e = delta_j - delta_i through
//                exact divided differences of s^-7, s^-4 and s^-1/2, so its
//                rounding error scales with |dF| instead of |F|.  A new FP64
//                reference is taken when max|delta| exceeds
//                min(ref_ratio * fmax, ref_dmax), and the convergence test
//                max_a |F_a| < tol is only ever passed on an FP64 evaluation.
//   FIRE state, positions, reductions and the final test are FP64 in both.
#include "minimize_launch.cuh"

namespace aqs {

size_t minimize_smem_bytes(int dim, int npc, int nrep, int nt, int cap, int mem) {
  return minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, mem);
}

int minimize_atoms_per_thread(int dim, int npc) {
  int apt = 0, threads = 0;
  choose_apt(dim, npc, &apt, &threads);
  return apt;
}

int minimize_staging(int dim, int npc, int nrep, int nt, int cap, int want) {
  return choose_mem(dim, npc, nrep, nt, cap, want);
}

int minimize_tpa(int npc, int want) { return effective_tpa(npc, want); }

bool minimize_launch_is_lean(int dim, int npc, int tpa) {
  return effective_tpa(npc, tpa) > 1 || minimize_is_lean(dim, minimize_atoms_per_thread(dim, npc));
}

static cudaError_t dispatch(int dim, bool mixed, const MinArgs* a, int n_clusters, int C, int npc,
                            int nrep, int nt, int cap, cudaStream_t s, int* max_clusters,
                            int staging, int tpa, bool gb = false) {
  int mem = choose_mem(dim, npc, nrep, nt, cap, staging);
  if (gb && mem != 0 && mem != 3)  // grid barriers read neighbour records from global memory
    mem = minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, 3) <= kSmemLimit ? 3 : 0;
  size_t smem = minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, mem);
  if (gb) {
    if (dim == 2)
      return mixed ? run_mem_2_mixed_gb(mem, a, n_clusters, C, npc, smem, s, max_clusters)
                   : run_mem_2_fp64_gb(mem, a, n_clusters, C, npc, smem, s, max_clusters);
    return mixed ? run_mem_3_mixed_gb(mem, a, n_clusters, C, npc, smem, s, max_clusters)
                 : run_mem_3_fp64_gb(mem, a, n_clusters, C, npc, smem, s, max_clusters);
  }
  if (effective_tpa(npc, tpa) == 2) {
    if (dim == 2)
      return mixed ? run_mem_2_mixed_t2(mem, a, n_clusters, C, npc, smem, s, max_clusters)
                   : run_mem_2_fp64_t2(mem, a, n_clusters, C, npc, smem, s, max_clusters);
    return mixed ? run_mem_3_mixed_t2(mem, a, n_clusters, C, npc, smem, s, max_clusters)
                 : run_mem_3_fp64_t2(mem, a, n_clusters, C, npc, smem, s, max_clusters);
  }
  if (dim == 2)
    return mixed ? run_mem_2_mixed(mem, a, n_clusters, C, npc, smem, s, max_clusters)
                 : run_mem_2_fp64(mem, a, n_clusters, C, npc, smem, s, max_clusters);
  return mixed ? run_mem_3_mixed(mem, a, n_clusters, C, npc, smem, s, max_clusters)
               : run_mem_3_fp64(mem, a, n_clusters, C, npc, smem, s, max_clusters);
}

cudaError_t launch_minimize(int dim, bool mixed, MinArgs a, int n_clusters, int C, int npc,
                            int nrep, int cap, cudaStream_t s, int staging, int tpa,
                            bool grid_barrier) {
  a.npc_launch = npc;
  a.nrep_launch = nrep;
  return dispatch(dim, mixed, &a, n_clusters, C, npc, nrep, a.nt, cap, s, nullptr, staging,
                  grid_barrier ? 1 : tpa, grid_barrier);
}

int minimize_max_grid_replicas(int dim, bool mixed, int C, int npc, int nrep, int nt, int cap,
                               int staging) {
  int m = 0;
  if (dispatch(dim, mixed, nullptr, 1, C, npc, nrep, nt, cap, nullptr, &m, staging, 1, true) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return m;
}

int minimize_max_active_clusters(int dim, bool mixed, int C, int npc, int nrep, int nt, int cap,
                                 int staging, int tpa) {
  int m = 0;
  if (dispatch(dim, mixed, nullptr, 1, C, npc, nrep, nt, cap, nullptr, &m, staging, tpa) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return m;
}

}  // namespace aqs
