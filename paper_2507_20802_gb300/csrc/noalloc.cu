// noalloc.cu -- FP64 energy, forces and shear stress of one configuration
// without any device allocation.
//
// Who needs this: code that runs where allocating device memory is not
// allowed or not possible -- for example a host callback or a plug-in that
// executes inside someone else's pre-planned memory budget, a process that
// shares a GPU under a strict allocation quota, or a caller holding a lock
// that cudaMalloc could deadlock against.  Such callers already own their
// input and output buffers; they only need the computation.  The regular path
// (aqs_create_system + aqs_energy_forces) allocates a system with Verlet lists
// and per-block scratch; this entry point instead walks all pairs and keeps its
// only scratch -- one partial energy and one partial virial per thread block --
// in a fixed array compiled into the library.
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// the library holds its 8 KiB until the process exits.  In host code its name
// is only a host-side stand-in, never a device address, so every call looks
// up the device address with cudaGetSymbolAddress in the caller's current
// context and passes it to the kernels.  The address belongs to a context, not
// to a device number (a reset device or another context has its own copy), so
// it is not cached; the lookup is a cheap host call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "aqs_internal.cuh"
#include "launch.cuh"

namespace aqs {

constexpr int kNoallocThreads = 128;
constexpr int kNoallocMaxBlocks = AQS_NOALLOC_MAX_ATOMS / kNoallocThreads;

// Partial sums (energy, virial) of each thread block of the last call.
static __device__ __align__(256) double g_noalloc_partial[2 * kNoallocMaxBlocks];

struct NoallocCoef {
  double A[AQS_MAX_TYPES * AQS_MAX_TYPES], B[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double C[AQS_MAX_TYPES * AQS_MAX_TYPES], rc2[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double e12[AQS_MAX_TYPES * AQS_MAX_TYPES], e6[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double Uc[AQS_MAX_TYPES * AQS_MAX_TYPES], dUc[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double rc[AQS_MAX_TYPES * AQS_MAX_TYPES];
  double H[9];
  int nt;
};

// All pairs, minimum image, one thread per atom i; tiles of j staged in
// shared memory.  Every pair is visited from both sides (energy and virial are
// halved by the final reduction).
template <int D>
__global__ void __launch_bounds__(kNoallocThreads) k_energy_all_pairs(
    const double* __restrict__ pos, const int32_t* __restrict__ types, int n, NoallocCoef cf,
    double* __restrict__ forces, double* __restrict__ partial) {
  __shared__ double sx[kNoallocThreads][D];
  __shared__ int st[kNoallocThreads];
  __shared__ double se[kNoallocThreads / 32], sw[kNoallocThreads / 32];
  const int i = blockIdx.x * kNoallocThreads + threadIdx.x;
  double xi[3] = {0.0, 0.0, 0.0}, F[3] = {0.0, 0.0, 0.0}, e = 0.0, w = 0.0;
  int ti = 0;
  if (i < n) {
    for (int c = 0; c < D; c++) xi[c] = pos[(int64_t)i * D + c];
    ti = types[i];
  }
  for (int j0 = 0; j0 < n; j0 += kNoallocThreads) {
    const int j = j0 + threadIdx.x;
    if (j < n) {
      for (int c = 0; c < D; c++) sx[threadIdx.x][c] = pos[(int64_t)j * D + c];
      st[threadIdx.x] = types[j];
    }
    __syncthreads();
    const int jn = min(kNoallocThreads, n - j0);
    if (i < n) {
      for (int jj = 0; jj < jn; jj++) {
        if (j0 + jj == i) continue;
        double d[3];
        for (int c = 0; c < D; c++) d[c] = sx[jj][c] - xi[c];
        min_image<D>(cf.H, d);
        double s = 0.0;
        for (int c = 0; c < D; c++) s += d[c] * d[c];
        const int k = ti * cf.nt + st[jj];
        if (s < cf.rc2[k]) {
          double u = 1.0 / s, ra = rsqrt(s);
          double u3 = u * u * u, u4 = u3 * u, u7 = u4 * u3;
          double phi = cf.A[k] * u7 + cf.B[k] * u4 + cf.C[k] * ra;
          for (int c = 0; c < D; c++) F[c] += phi * d[c];
          double r = s * ra;
          e += cf.e12[k] * u3 * u3 - cf.e6[k] * u3 - cf.Uc[k] - (r - cf.rc[k]) * cf.dUc[k];
          w += phi * d[0] * d[1];
        }
      }
    }
    __syncthreads();
  }
  if (i < n)
    for (int c = 0; c < D; c++) forces[(int64_t)i * D + c] = F[c];
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = e;
    sw[threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, tw = 0.0;
    for (int k = 0; k < kNoallocThreads / 32; k++) {
      te += se[k];
      tw += sw[k];
    }
    partial[2 * blockIdx.x] = te;
    partial[2 * blockIdx.x + 1] = tw;
  }
}

// Sums the block partials in block order (deterministic) into
// energy_tau[0] = E and energy_tau[1] = tau.
__global__ void k_energy_finish(const double* __restrict__ partial, int nblocks, double inv_vol,
                                double* __restrict__ energy_tau) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e = 0.0, w = 0.0;
  for (int b = 0; b < nblocks; b++) {
    e += partial[2 * b];
    w += partial[2 * b + 1];
  }
  energy_tau[0] = 0.5 * e;
  energy_tau[1] = 0.5 * w * inv_vol;
}

// Device address of g_noalloc_partial in the current context.
static cudaError_t noalloc_scratch(void** out) {
  *out = nullptr;
  return cudaGetSymbolAddress(out, g_noalloc_partial);
}

}  // namespace aqs

using namespace aqs;

extern "C" aqs_status aqs_energy_forces_noalloc(int dim, int64_t n, const double* pos,
                                                const int32_t* types, const double* box,
                                                const aqs_potential* pot, double* forces,
                                                double* energy_tau, void* stream) {
  if (dim != 2 && dim != 3) return AQS_ERR_INVALID_ARG;
  if (!pos || !types || !box || !pot || !forces || !energy_tau) return AQS_ERR_INVALID_ARG;
  if (n < 2 || n > AQS_NOALLOC_MAX_ATOMS) {
    fprintf(stderr,
            "aqs_energy_forces_noalloc: %lld atoms is outside the supported range [2, %d] "
            "(the fixed scratch array holds one partial sum per %d atoms)\n",
            (long long)n, AQS_NOALLOC_MAX_ATOMS, kNoallocThreads);
    return AQS_ERR_INVALID_ARG;
  }
  const int nt = pot->n_types;
  if (nt < 1 || nt > AQS_MAX_TYPES || !(pot->rc_factor > 0.0)) return AQS_ERR_INVALID_ARG;
  NoallocCoef cf;
  cf.nt = nt;
  double rcmax = 0.0;
  for (int a = 0; a < nt; a++)
    for (int b = 0; b < nt; b++) {
      const int k = a * nt + b;
      const double sig = pot->sigma[k], eps = pot->eps[k];
      if (!(sig > 0.0) || !(eps >= 0.0)) return AQS_ERR_INVALID_ARG;
      const double rc = pot->rc_factor * sig;
      const double s6 = std::pow(sig, 6.0);
      const double src = sig / rc, src2 = src * src, src6 = src2 * src2 * src2;
      const double uc = 4.0 * eps * (src6 * src6 - src6);
      const double duc = -24.0 * eps * (2.0 * src6 * src6 - src6) / rc;
      cf.A[k] = -48.0 * eps * s6 * s6;
      cf.B[k] = 24.0 * eps * s6;
      cf.C[k] = -duc;
      cf.rc2[k] = rc * rc;
      cf.e12[k] = 4.0 * eps * s6 * s6;
      cf.e6[k] = 4.0 * eps * s6;
      cf.Uc[k] = uc;
      cf.dUc[k] = duc;
      cf.rc[k] = rc;
      rcmax = std::fmax(rcmax, rc);
    }
  for (int k = 0; k < 9; k++) cf.H[k] = k < dim * dim ? box[k] : 0.0;
  // upper-triangular cell with positive diagonal and a tilt in H[0][1] only
  // (the width test below and the minimum image assume it); the cutoff below
  // half of the smallest perpendicular width
  for (int a = 0; a < dim; a++) {
    if (!(box[a * dim + a] > 0.0)) return AQS_ERR_INVALID_ARG;
    for (int b = 0; b < a; b++)
      if (box[a * dim + b] != 0.0) return AQS_ERR_INVALID_ARG;
  }
  if (dim == 3 && (box[2] != 0.0 || box[5] != 0.0)) return AQS_ERR_INVALID_ARG;
  const double ly = box[1 * dim + 1], t = box[0 * dim + 1];
  double wmin = std::fmin(box[0] / std::sqrt(1.0 + (t / ly) * (t / ly)), ly);
  if (dim == 3) wmin = std::fmin(wmin, box[8]);
  if (!(2.0 * rcmax < wmin)) return AQS_ERR_BOX_TOO_SMALL;
  const double vol = dim == 2 ? box[0] * box[3] : box[0] * box[4] * box[8];

  void* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return AQS_ERR_CUDA;
  }
  double* partial = static_cast<double*>(scratch);
  const int nblocks = (int)((n + kNoallocThreads - 1) / kNoallocThreads);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  count_launch();
  if (dim == 2)
    k_energy_all_pairs<2><<<nblocks, kNoallocThreads, 0, s>>>(pos, types, (int)n, cf, forces, partial);
  else
    k_energy_all_pairs<3><<<nblocks, kNoallocThreads, 0, s>>>(pos, types, (int)n, cf, forces, partial);
  count_launch();
  k_energy_finish<<<1, 32, 0, s>>>(partial, nblocks, 1.0 / vol, energy_tau);
  if (cudaGetLastError() != cudaSuccess) return AQS_ERR_CUDA;
  return AQS_OK;
}
