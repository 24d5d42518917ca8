// minimize.cuh -- arguments and launcher of the persistent FIRE minimiser.
#pragma once
#include "aqs_internal.cuh"

namespace aqs {

struct MinArgs {
  const RepGeom* geom;
  RepState* state;
  const int* work;  // replica index per cluster
  double* x;        // [D][ntot]; holds x_ref inside a launch in mixed mode
  double* v;        // [D][ntot]
  double* fref;     // [D][ntot] (mixed)
  double* dl;       // [D][ntot] delta (mixed)
  double* xs;       // [D][ntot] positions at the start of the minimisation
  double* xb;       // [D][ntot] positions at the last list build (affinely mapped)
  const int32_t* type;
  int32_t* cell;
  uint32_t* nb;
  int32_t* nnb;
  // in-kernel Verlet rebuild (without re-sorting the atoms): scratch per cell
  // (count, cstart at the replica's cell_off) and per atom (cellatoms)
  int32_t* count;
  int32_t* cstart;
  int32_t* cellatoms;
  int cap;                // list capacity per atom
  int inkernel_rebuild;   // 1: rebuild lists inside the kernel when the skin trips
  float rl2f[AQS_MAX_TYPES * AQS_MAX_TYPES];
  const PairCoef* coef;
  int64_t ntot;
  int nt;
  FireDev fire;
  double skin, rlist;
  int64_t launch_budget;  // FIRE iterations per launch before yielding
  double* rec;            // [R][rec_stride][5] per-step records (nullable)
  int64_t rec_stride;
  double* snap;           // [R][snap_stride] caller-order positions after step 0 (nullable)
  int64_t snap_stride;
  const int32_t* perm;    // [ntot] caller index of every atom
  const float* warm_u;    // [ntot][D] learned start displacement per unit strain, caller order
                          // within each replica (nullable)
  int npc_launch;         // shared-memory stride (largest npc of the launch)
  int nrep_launch;        // largest replica of the launch (staged positions)
  // [ntot] position records in global memory (Pub<D>, 16 B in 2D, 32 B in 3D),
  // the source of neighbour records in staging modes 0 and 3
  void* pubg;
  // per-atom state of launches with 4 or 8 atoms per thread (allocated on
  // first use): [5][3][ntot] FP32 (q_ref, delta, v, f_ref, f_used) and
  // [3][ntot] FP64 force
  float* lean32;
  double* lean64;
  // deformation history (nullable): [R][hist_stride][kHistFields], the map
  // and cell of every job step (step 0 of a no-affine job unused); with it
  // the kernel keeps the full cell in RepState::Hc / Hb
  const double* hist;
  int64_t hist_stride;
  // grid-barrier launches (cooperative, no clusters): CTAs per replica,
  // reduction partials [R][16][kNumRed], barrier words [R][2] (read as one
  // 64-bit arrival counter per replica, 8-byte aligned, zeroed before every
  // launch), error word (set when a barrier wait runs out)
  int gb_C;
  double* gb_part;
  unsigned* gb_bar;
  int* gb_err;
};

// Staging modes of the minimiser (where a CTA finds list rows and the
// published position records of its neighbours):
//   0: rows read from global memory each iteration, records from global memory
//   1: rows staged in shared memory, records read from the owner CTA (DSMEM)
//   2: rows staged, records of the whole replica copied into shared memory
//      from the owner CTAs each iteration
//   3: rows staged, records from global memory
// All modes read bitwise identical values, so they give identical results.
constexpr int kNumStaging = 4;

size_t minimize_smem_bytes(int dim, int npc, int nrep, int nt, int cap, int mem);
// staging mode used for this configuration: `want` if it fits in shared
// memory (want in 0..3), else the automatic choice (2, then 1, then 0)
int minimize_staging(int dim, int npc, int nrep, int nt, int cap, int want);
// tpa: threads per atom of the force phase wanted (1, or 2 where npc * 2
// threads fit in a CTA; see minimize_tpa)
cudaError_t launch_minimize(int dim, bool mixed, MinArgs a, int n_clusters, int C, int npc,
                            int nrep, int cap, cudaStream_t s, int staging = -1, int tpa = 1,
                            bool grid_barrier = false);
// grid-barrier launches: how many replicas of C CTAs fit the device at once
// (cooperative launches need every CTA resident)
int minimize_max_grid_replicas(int dim, bool mixed, int C, int npc, int nrep, int nt, int cap,
                               int staging);
// threads per atom a launch with npc atoms per CTA uses when `want` is asked
int minimize_tpa(int npc, int want);
// the launch keeps per-atom state in MinArgs::lean32 / lean64
bool minimize_launch_is_lean(int dim, int npc, int tpa);
// atoms per thread of a launch with npc atoms per CTA (1, 2, 4 or 8; lean
// launches use up to 1024 threads, the others up to 512)
int minimize_atoms_per_thread(int dim, int npc);
// launches that keep the per-atom state in MinArgs::lean32 / lean64 instead
// of registers (where registers would spill)
constexpr bool minimize_is_lean(int dim, int apt) { return apt >= 4 || (dim == 3 && apt >= 2); }
// clusters of C CTAs that can be resident at once for this configuration
int minimize_max_active_clusters(int dim, bool mixed, int C, int npc, int nrep, int nt, int cap,
                                 int staging = -1, int tpa = 1);

}  // namespace aqs
