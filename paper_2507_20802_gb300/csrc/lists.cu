// lists.cu -- cell binning by sorted cell key and Verlet-list construction
// under Lees-Edwards (sheared) periodic boundaries.
//
// Cells live on the fractional-coordinate grid s = H^-1 r in [0,1)^d, so they
// shear with the cell and the 3^d stencil is complete as long as every
// perpendicular cell width is at least rc_max + skin (checked on the host).
// Rebuild pipeline for the replicas whose flag is set:
//   k_bin       wrap positions by whole lattice vectors, cell key, histogram
//   k_scan      exclusive scan of the cell counts (one CTA per replica)
//   k_scatter   counting-sort scatter
//   k_cellsort  insertion sort inside each cell by previous index, which makes
//               the order (and every later floating-point sum) deterministic
//   k_permute / k_copyback   gather all per-atom arrays into the new order
//   k_verlet    full neighbour list within rc_ab + skin, column-major
#include <math.h>

#include "aqs_internal.cuh"
#include "launch.cuh"
#include "lists.cuh"

namespace aqs {

template <int D>
__global__ void k_bin(BuildArgs a) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= a.ntot) return;
  int r = a.rep_of[gi];
  if (!a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  const int64_t N = a.ntot;
  double x[3], s[3];
  for (int c = 0; c < D; c++) x[c] = a.x[c * N + gi];
  // back substitution of the upper-triangular H s = x
  for (int c = D - 1; c >= 0; c--) {
    double t = x[c];
    for (int k = c + 1; k < D; k++) t -= g.H[c * D + k] * s[k];
    s[c] = t / g.H[c * D + c];
  }
  double n[3];
  for (int c = 0; c < D; c++) n[c] = floor(s[c]);
  for (int c = 0; c < D; c++) {
    double sh = 0.0;
    for (int k = c; k < D; k++) sh += g.H[c * D + k] * n[k];
    if (sh != 0.0) a.x[c * N + gi] = x[c] - sh;
  }
  int key = 0, mul = 1;
  for (int c = 0; c < D; c++) {
    int ic = (int)floor((s[c] - n[c]) * g.nc[c]);
    ic = ic < 0 ? 0 : (ic >= g.nc[c] ? g.nc[c] - 1 : ic);
    key += ic * mul;
    mul *= g.nc[c];
  }
  a.key[gi] = key;
  atomicAdd(&a.count[g.cell_off + key], 1);
}

__global__ void k_scan(BuildArgs a) {
  int r = blockIdx.x;
  if (!a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  __shared__ int carry;
  __shared__ int wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < g.ncell; base += blockDim.x) {
    int c = base + threadIdx.x;
    int v = c < g.ncell ? a.count[g.cell_off + c] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < nw) wsum[lane] = ws;
    }
    __syncthreads();
    int excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - v;
    if (c < g.ncell) {
      a.cstart[g.cell_off + c] = excl;
      a.count[g.cell_off + c] = 0;  // reused as the scatter cursor
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.cstart[g.cell_off + g.ncell] = carry;
}

__global__ void k_scatter(BuildArgs a) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= a.ntot) return;
  int r = a.rep_of[gi];
  if (!a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  int c = g.cell_off + a.key[gi];
  int p = a.cstart[c] + atomicAdd(&a.count[c], 1);
  a.order[g.off + p] = gi;
}

// one thread per cell; sort the cell's slice of `order` by previous index
__global__ void k_cellsort(BuildArgs a, int total_cells) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= total_cells) return;
  int r = a.cell_rep[c];
  if (r < 0 || !a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  int lc = c - g.cell_off;
  if (lc >= g.ncell) return;
  int64_t b = g.off + a.cstart[c], e = g.off + a.cstart[c + 1];
  for (int64_t i = b + 1; i < e; i++) {
    int64_t v = a.order[i];
    int64_t j = i - 1;
    while (j >= b && a.order[j] > v) {
      a.order[j + 1] = a.order[j];
      j--;
    }
    a.order[j + 1] = v;
  }
}

template <int D>
__global__ void k_permute(BuildArgs a) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.ntot) return;
  int r = a.rep_of[p];
  if (!a.flag[r]) return;
  const int64_t N = a.ntot;
  int64_t o = a.order[p];
  for (int c = 0; c < D; c++) {
    a.tmp[(0 * D + c) * N + p] = a.x[c * N + o];
    a.tmp[(1 * D + c) * N + p] = a.v[c * N + o];
    a.tmp[(2 * D + c) * N + p] = a.xs[c * N + o];
  }
  a.itmp[0 * N + p] = a.type[o];
  a.itmp[1 * N + p] = a.perm[o];
  a.itmp[2 * N + p] = a.key[o];
}

template <int D>
__global__ void k_copyback(BuildArgs a) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.ntot) return;
  int r = a.rep_of[p];
  if (!a.flag[r]) return;
  const int64_t N = a.ntot;
  for (int c = 0; c < D; c++) {
    a.x[c * N + p] = a.tmp[(0 * D + c) * N + p];
    a.v[c * N + p] = a.tmp[(1 * D + c) * N + p];
    a.xs[c * N + p] = a.tmp[(2 * D + c) * N + p];
    a.xb[c * N + p] = a.x[c * N + p];
  }
  a.type[p] = a.itmp[0 * N + p];
  int u = a.itmp[1 * N + p];
  a.perm[p] = u;
  a.cell[p] = a.itmp[2 * N + p];
  a.inv[a.geom[r].off + u] = (int32_t)(p - a.geom[r].off);
}

template <int D>
__global__ void k_verlet(BuildArgs a) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= a.ntot) return;
  int r = a.rep_of[gi];
  if (!a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  const int64_t N = a.ntot;
  const int il = (int)(gi - g.off);
  const int ci = a.cell[gi];
  int cc[3] = {ci % g.nc[0], (ci / g.nc[0]) % g.nc[1], D == 3 ? ci / (g.nc[0] * g.nc[1]) : 0};
  double oi[3];
  cell_origin<D>(g.H, g.nc, ci, oi);
  float qi[3];
  for (int c = 0; c < D; c++) qi[c] = (float)(a.x[c * N + gi] - oi[c]);
  const int ti = a.type[gi];
  int cnt = 0;
  const int zlo = D == 3 ? -1 : 0, zhi = D == 3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; dz++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dx = -1; dx <= 1; dx++) {
        int nx = (cc[0] + dx + g.nc[0]) % g.nc[0];
        int ny = (cc[1] + dy + g.nc[1]) % g.nc[1];
        int nz = D == 3 ? (cc[2] + dz + g.nc[2]) % g.nc[2] : 0;
        int cj = nx + g.nc[0] * (ny + g.nc[1] * nz);
        int code = (dx + 1) + 3 * (dy + 1) + (D == 3 ? 9 * (dz + 1) : 0);
        double of[3], oj[3];
        cell_offset<D>(g.H, g.nc, code, of);
        cell_origin<D>(g.H, g.nc, cj, oj);
        float off32[3];
        for (int c = 0; c < D; c++) off32[c] = (float)of[c];
        int b = a.cstart[g.cell_off + cj], e = a.cstart[g.cell_off + cj + 1];
        for (int jl = b; jl < e; jl++) {
          int64_t gj = g.off + jl;
          if (gj == gi) continue;
          float s = 0.0f;
          for (int c = 0; c < D; c++) {
            float d = ((float)(a.x[c * N + gj] - oj[c]) - qi[c]) + off32[c];
            s = fmaf(d, d, s);
          }
          int tj = a.type[gj];
          if (s < a.rl2f[ti * a.nt + tj]) {
            if (cnt < a.cap)
              a.nb[g.nb_off + (int64_t)cnt * g.n + il] = encode_nb(jl % g.npc, jl / g.npc, code, tj);
            cnt++;
          }
        }
      }
  a.nnb[gi] = cnt < a.cap ? cnt : a.cap;
  if (cnt > a.cap) atomicMax(&a.overflow[r], cnt);
}

// total list length of each rebuilt replica (one CTA per replica)
__global__ void k_sum_nnb(BuildArgs a, int64_t* out) {
  int r = blockIdx.x;
  if (!a.flag[r]) return;
  const RepGeom& g = a.geom[r];
  int64_t t = 0;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) t += a.nnb[g.off + i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ int64_t ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += ws[w];
    out[r] = s;
  }
}

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

cudaError_t launch_sum_nnb(const BuildArgs& a, int n_rep, int64_t* out, cudaStream_t s) {
  count_launch();
  k_sum_nnb<<<n_rep, 256, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t launch_rebuild_bin(int dim, const BuildArgs& a, int n_rep, cudaStream_t s) {
  const int T = 256;
  count_launch();
  if (dim == 2) k_bin<2><<<nblk(a.ntot, T), T, 0, s>>>(a);
  else k_bin<3><<<nblk(a.ntot, T), T, 0, s>>>(a);
  count_launch();
  k_scan<<<n_rep, 1024, 0, s>>>(a);
  count_launch();
  k_scatter<<<nblk(a.ntot, T), T, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rebuild_sort(int dim, const BuildArgs& a, int total_cells, cudaStream_t s) {
  const int T = 256;
  count_launch();
  k_cellsort<<<nblk(total_cells, T), T, 0, s>>>(a, total_cells);
  count_launch();
  if (dim == 2) k_permute<2><<<nblk(a.ntot, T), T, 0, s>>>(a);
  else k_permute<3><<<nblk(a.ntot, T), T, 0, s>>>(a);
  count_launch();
  if (dim == 2) k_copyback<2><<<nblk(a.ntot, T), T, 0, s>>>(a);
  else k_copyback<3><<<nblk(a.ntot, T), T, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rebuild_verlet(int dim, const BuildArgs& a, cudaStream_t s) {
  const int T = 128;
  count_launch();
  if (dim == 2) k_verlet<2><<<nblk(a.ntot, T), T, 0, s>>>(a);
  else k_verlet<3><<<nblk(a.ntot, T), T, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace aqs
