// lists.cuh -- arguments and launchers of the cell/Verlet list build.
#pragma once
#include "aqs_internal.cuh"

namespace aqs {

struct BuildArgs {
  const RepGeom* geom;
  const int32_t* rep_of;    // [ntot] replica of each atom
  const uint8_t* flag;      // [R] rebuild this replica?
  double* x;                // [D][ntot]
  double* v;                // [D][ntot]
  double* xs;               // [D][ntot]
  double* xb;               // [D][ntot]
  int32_t* type;            // [ntot]
  int32_t* perm;            // [ntot] sorted -> caller index (replica-local)
  int32_t* inv;             // [ntot] caller index -> sorted (replica-local)
  int32_t* cell;            // [ntot] replica-local cell of each atom
  int32_t* key;             // [ntot] scratch: cell key before sorting
  int64_t* order;           // [ntot] scratch: new position -> old global index
  int32_t* count;           // [total cells] histogram / scatter cursor
  int32_t* cstart;          // [total cells] cell start (replica-local atom index)
  const int32_t* cell_rep;  // [total cells] replica of each global cell slot
  double* tmp;              // [3 D][ntot] scratch
  int32_t* itmp;            // [3][ntot] scratch
  uint32_t* nb;             // neighbour entries
  int32_t* nnb;             // [ntot] neighbours per atom
  int32_t* overflow;        // [R] largest neighbour count above capacity
  float rl2f[AQS_MAX_TYPES * AQS_MAX_TYPES];  // (rc_ab + skin)^2 plus a rounding margin
  int nt;
  int cap;
  int64_t ntot;
};

cudaError_t launch_rebuild_bin(int dim, const BuildArgs& a, int n_rep, cudaStream_t s);
cudaError_t launch_rebuild_sort(int dim, const BuildArgs& a, int total_cells, cudaStream_t s);
cudaError_t launch_rebuild_verlet(int dim, const BuildArgs& a, cudaStream_t s);
cudaError_t launch_sum_nnb(const BuildArgs& a, int n_rep, int64_t* out, cudaStream_t s);

}  // namespace aqs
