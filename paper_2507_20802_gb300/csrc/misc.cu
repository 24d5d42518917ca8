// misc.cu -- the O(N) kernels around the minimiser: affine simple shear,
// level-I replication of r_star, user-order gather/scatter, the equality /
// non-affine displacement test and a list-based FP64 energy evaluation.
#include <math.h>

#include "aqs_internal.cuh"
#include "launch.cuh"
#include "misc.cuh"

namespace aqs {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Simple shear F^(dgamma) (Sec. 2.1 Eqs. 2-3, Eq. 16): x += dgamma y.  The
// list-build reference positions xb follow the same map, so the skin test only
// sees non-affine motion plus the bounded affine change of short pair vectors.
__global__ void k_affine(double* x, double* xb, const int32_t* rep_of, const double* dg,
                         int64_t N) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double g = dg[rep_of[i]];
  if (g == 0.0) return;
  x[i] = fma(g, x[N + i], x[i]);
  xb[i] = fma(g, xb[N + i], xb[i]);
}

cudaError_t launch_affine(double* x, double* xb, const int32_t* rep_of, const double* dg,
                          int64_t N, cudaStream_t s) {
  count_launch();
  k_affine<<<nblk(N, 256), 256, 0, s>>>(x, xb, rep_of, dg, N);
  return cudaGetLastError();
}

// Deformation-history increment (Eqs. 1-3 with a general matrix, expressed in
// the frame where the cell stays upper triangular): r <- M r, r_b <- M r_b.
// The diagonal term first, so that simple shear is the fma of k_affine.
__device__ __forceinline__ void map_upper(int D, const double* M, const double* v, double* out) {
  for (int a = 0; a < D; a++) {
    double s = M[a * 3 + a] * v[a];
    for (int c = a + 1; c < D; c++) s = fma(M[a * 3 + c], v[c], s);
    out[a] = s;
  }
}

__global__ void k_deform(int D, double* x, double* xb, const int32_t* rep_of, const uint8_t* flag,
                         const double* maps, int64_t N) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int r = rep_of[i];
  if (!flag[r]) return;
  const double* M = maps + 9 * (int64_t)r;
  double v[3], w[3];
  for (int c = 0; c < D; c++) v[c] = x[c * N + i];
  map_upper(D, M, v, w);
  for (int c = 0; c < D; c++) x[c * N + i] = w[c];
  for (int c = 0; c < D; c++) v[c] = xb[c * N + i];
  map_upper(D, M, v, w);
  for (int c = 0; c < D; c++) xb[c * N + i] = w[c];
}

cudaError_t launch_deform(int dim, double* x, double* xb, const int32_t* rep_of,
                          const uint8_t* flag, const double* maps, int64_t N, cudaStream_t s) {
  count_launch();
  k_deform<<<nblk(N, 256), 256, 0, s>>>(dim, x, xb, rep_of, flag, maps, N);
  return cudaGetLastError();
}

// Level I (Sec. 3.2, Eq. 18): copies of one replica, copy c sheared by
// shift[c] (= c K dgamma), or mapped by maps[c] under a deformation history;
// FIRE velocities cleared.
__global__ void k_copy_rep(RepCopy a) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)a.ncopy * a.n) return;
  int c = (int)(idx / a.n);
  int p = (int)(idx % a.n);
  int64_t si = a.soff + p, di = a.doff[c] + p;
  if (a.maps) {
    double v[3], w[3];
    const double* M = a.maps + 9 * (int64_t)c;
    for (int k = 0; k < a.D; k++) v[k] = a.sx[k * a.sN + si];
    map_upper(a.D, M, v, w);
    for (int k = 0; k < a.D; k++) a.dx[k * a.dN + di] = w[k];
    for (int k = 0; k < a.D; k++) v[k] = a.sxb[k * a.sN + si];
    map_upper(a.D, M, v, w);
    for (int k = 0; k < a.D; k++) {
      a.dxb[k * a.dN + di] = w[k];
      a.dv[k * a.dN + di] = 0.0;
    }
  } else {
    double g = a.shift[c];
    for (int k = 0; k < a.D; k++) {
      double xv = a.sx[k * a.sN + si], bv = a.sxb[k * a.sN + si];
      if (k == 0 && g != 0.0) {
        xv = fma(g, a.sx[a.sN + si], xv);
        bv = fma(g, a.sxb[a.sN + si], bv);
      }
      a.dx[k * a.dN + di] = xv;
      a.dxb[k * a.dN + di] = bv;
      a.dv[k * a.dN + di] = 0.0;
    }
  }
  a.dtype[di] = a.stype[si];
  a.dperm[di] = a.sperm[si];
  a.dinv[di] = a.sinv[si];
  a.dcell[di] = a.scell[si];
  a.dnnb[di] = a.snnb[si];
}

__global__ void k_copy_nb(RepCopy a) {
  int64_t per = (int64_t)a.cap * a.n;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= per * a.ncopy) return;
  int c = (int)(idx / per);
  int64_t k = idx % per;
  a.dnb[a.dnb_off[c] + k] = a.snb[a.snb_off + k];
}

cudaError_t launch_copy_rep(const RepCopy& a, cudaStream_t s) {
  if (a.ncopy <= 0 || a.n <= 0) return cudaSuccess;
  count_launch();
  k_copy_rep<<<nblk((int64_t)a.ncopy * a.n, 256), 256, 0, s>>>(a);
  if (a.cap > 0) {
    count_launch();
    k_copy_nb<<<nblk((int64_t)a.ncopy * a.cap * a.n, 256), 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// caller order <-> internal order
__global__ void k_gather_user(const double* x, int64_t N, int64_t off, int n, const int32_t* perm,
                              int D, double* out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int u = perm[off + p];
  for (int c = 0; c < D; c++) out[(int64_t)u * D + c] = x[c * N + off + p];
}

__global__ void k_scatter_user(const double* in, double* x, int64_t N, int64_t off, int n,
                               const int32_t* perm, int D) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int u = perm[off + p];
  for (int c = 0; c < D; c++) x[c * N + off + p] = in[(int64_t)u * D + c];
}

cudaError_t launch_gather_user(const double* x, int64_t N, int64_t off, int n, const int32_t* perm,
                               int D, double* out, cudaStream_t s) {
  count_launch();
  k_gather_user<<<nblk(n, 256), 256, 0, s>>>(x, N, off, n, perm, D, out);
  return cudaGetLastError();
}

cudaError_t launch_scatter_user(const double* in, double* x, int64_t N, int64_t off, int n,
                                const int32_t* perm, int D, cudaStream_t s) {
  count_launch();
  k_scatter_user<<<nblk(n, 256), 256, 0, s>>>(in, x, N, off, n, perm, D);
  return cudaGetLastError();
}

// Equality test of Eq. 20 / non-affine displacement: for one pair of
// configurations (a, b) at the same cell H,
//   m = max_i | mi(a_i - b_i) - mean_j mi(a_j - b_j) |.
// One CTA per pair, two passes, fixed-order block reductions.
template <int D>
__global__ void k_compare(const CmpJob* jobs, double* out) {
  const CmpJob& J = jobs[blockIdx.x];
  __shared__ double sm[32][3];
  __shared__ double mean[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < J.n; i += blockDim.x) {
    double d[3];
    for (int c = 0; c < D; c++) d[c] = J.a[i * J.sa + c * J.sc] - J.b[i * J.sb + c * J.sc2];
    min_image<D>(J.H, d);
    for (int c = 0; c < D; c++) acc[c] += d[c];
  }
  for (int c = 0; c < D; c++) {
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0) sm[warp][c] = acc[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < D; c++) {
      double t = 0.0;
      for (int w = 0; w < nw; w++) t += sm[w][c];
      mean[c] = t / J.n;
    }
  }
  __syncthreads();
  double m = 0.0;
  for (int i = threadIdx.x; i < J.n; i += blockDim.x) {
    double d[3], s = 0.0;
    for (int c = 0; c < D; c++) d[c] = J.a[i * J.sa + c * J.sc] - J.b[i * J.sb + c * J.sc2];
    min_image<D>(J.H, d);
    for (int c = 0; c < D; c++) s += (d[c] - mean[c]) * (d[c] - mean[c]);
    m = fmax(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if (lane == 0) sm[warp][0] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; w++) t = fmax(t, sm[w][0]);
    out[blockIdx.x] = sqrt(t);
  }
}

cudaError_t launch_compare(int dim, const CmpJob* jobs, int njobs, double* out, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  count_launch();
  if (dim == 2) k_compare<2><<<njobs, 256, 0, s>>>(jobs, out);
  else k_compare<3><<<njobs, 256, 0, s>>>(jobs, out);
  return cudaGetLastError();
}

// FP64 energy, forces and stress of one replica from its Verlet list, reading
// positions from global memory.  Forces go out in caller order; per-block
// partial sums of E and of the virial are summed on the host in block order.
template <int D>
__global__ void k_energy(EnergyArgs a) {
  const RepGeom& g = *a.geom;
  const int64_t N = a.ntot;
  int il = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0, w = 0.0;
  if (il < g.n) {
    int64_t gi = g.off + il;
    double oi[3], qi[3], F[3] = {0.0, 0.0, 0.0};
    cell_origin<D>(g.H, g.nc, a.cell[gi], oi);
    for (int c = 0; c < D; c++) qi[c] = a.x[c * N + gi] - oi[c];
    int ti = a.type[gi];
    int nn = a.nnb[gi];
    for (int j = 0; j < nn; j++) {
      uint32_t ent = a.nb[g.nb_off + (int64_t)j * g.n + il];
      int jl = nb_owner(ent) * g.npc + nb_slot(ent);
      int64_t gj = g.off + jl;
      double oj[3], of[3], d[3];
      cell_origin<D>(g.H, g.nc, a.cell[gj], oj);
      cell_offset<D>(g.H, g.nc, nb_code(ent), of);
      double s = 0.0;
      for (int c = 0; c < D; c++) {
        d[c] = ((a.x[c * N + gj] - oj[c]) - qi[c]) + of[c];
        s += d[c] * d[c];
      }
      const PairCoef& cf = a.coef[ti * a.nt + nb_type(ent)];
      if (s < cf.rc2) {
        double u = 1.0 / s, ra = rsqrt(s);
        double u3 = u * u * u, u4 = u3 * u, u7 = u4 * u3;
        double phi = cf.A * u7 + cf.B * u4 + cf.C * ra;
        for (int c = 0; c < D; c++) F[c] += phi * d[c];
        double r = s * ra;
        e += cf.e12 * u3 * u3 - cf.e6 * u3 - cf.Uc - (r - cf.rc) * cf.dUc;
        w += phi * d[0] * d[1];
      }
    }
    if (a.forces) {
      int u = a.perm[gi];
      for (int c = 0; c < D; c++) a.forces[(int64_t)u * D + c] = F[c];
    }
  }
  __shared__ double se[32], sw[32];
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    se[warp] = e;
    sw[warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, tw = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      te += se[k];
      tw += sw[k];
    }
    a.partial[2 * blockIdx.x] = te;
    a.partial[2 * blockIdx.x + 1] = tw;
  }
}

int energy_blocks(int n) { return nblk(n, 128); }

cudaError_t launch_energy(int dim, const EnergyArgs& a, int n, cudaStream_t s) {
  count_launch();
  if (dim == 2) k_energy<2><<<energy_blocks(n), 128, 0, s>>>(a);
  else k_energy<3><<<energy_blocks(n), 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace aqs
