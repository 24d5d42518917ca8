// misc.cuh -- arguments and launchers of the O(N) helper kernels.
#pragma once
#include "aqs_internal.cuh"

namespace aqs {

struct RepCopy {
  const double *sx, *sxb;
  const int32_t *stype, *sperm, *sinv, *scell, *snnb;
  const uint32_t* snb;
  int64_t sN, soff, snb_off;
  double *dx, *dxb, *dv;
  int32_t *dtype, *dperm, *dinv, *dcell, *dnnb;
  uint32_t* dnb;
  int64_t dN;
  const int64_t* doff;     // device [ncopy]
  const int64_t* dnb_off;  // device [ncopy]
  const double* shift;     // device [ncopy]
  // device [ncopy][9] (nullable): instead of the shear shift, copy c is mapped
  // by the upper-triangular matrix maps[c] (row-major 3 x 3 slots)
  const double* maps;
  int n, cap, ncopy, D;
};

// element i, component c of a is a[i * sa + c * sc] (same for b with sb, sc2)
struct CmpJob {
  const double* a;
  const double* b;
  int64_t sa, sc, sb, sc2;
  double H[9];
  int n;
};

struct EnergyArgs {
  const RepGeom* geom;  // the replica's geometry (device)
  const double* x;
  const int32_t* type;
  const int32_t* cell;
  const int32_t* perm;
  const uint32_t* nb;
  const int32_t* nnb;
  const PairCoef* coef;
  double* forces;   // caller order, nullable
  double* partial;  // [2 * blocks]
  int64_t ntot;
  int nt;
};

cudaError_t launch_affine(double* x, double* xb, const int32_t* rep_of, const double* dg,
                          int64_t N, cudaStream_t s);
cudaError_t launch_copy_rep(const RepCopy& a, cudaStream_t s);
// General affine increment of a deformation history: atoms of replica r (and
// their list-build positions) are mapped by the upper-triangular maps[r]
// (device [R][9], row-major 3 x 3 slots); replicas with flag[r] == 0 untouched.
cudaError_t launch_deform(int dim, double* x, double* xb, const int32_t* rep_of,
                          const uint8_t* flag, const double* maps, int64_t N, cudaStream_t s);
cudaError_t launch_gather_user(const double* x, int64_t N, int64_t off, int n, const int32_t* perm,
                               int D, double* out, cudaStream_t s);
cudaError_t launch_scatter_user(const double* in, double* x, int64_t N, int64_t off, int n,
                                const int32_t* perm, int D, cudaStream_t s);
cudaError_t launch_compare(int dim, const CmpJob* jobs, int njobs, double* out, cudaStream_t s);
int energy_blocks(int n);
cudaError_t launch_energy(int dim, const EnergyArgs& a, int n, cudaStream_t s);

}  // namespace aqs
