// warm.cu -- learned warm start: per-atom neighbour-shell features and a
// small per-atom MLP (input -> 128 -> 128 -> 128 -> dim, GELU), run and
// trained on tensor cores in BF16 with FP32 accumulation.
//
// The paper leaves faster starting points for the minimiser as future work
// (Sec. 5).  Here the network predicts each atom's non-affine displacement per
// unit strain u_i for the next increment; the minimisation starts from
// F^(dgamma) r_k + dgamma u and FIRE still decides the minimum.
//
// Tensor-core tiles use mma.sync.aligned.m16n8k16 (BF16 in, FP32 out) with the
// operand layouts of the PTX ISA.  A CTA handles 32 rows (2 warps x 16 rows);
// weights live in shared memory as BF16, K contiguous.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "aqs_internal.cuh"
#include "launch.cuh"
#include "warm.cuh"

namespace aqs {

// ---------------------------------------------------------------- features
// Features of atom i: displacements d_ij = mi(r_j - r_i) of its NB nearest
// atoms sorted by (|d|^2, caller index j), then a one-hot species code.  The
// arithmetic (difference, minimum image from the last axis to the first,
// sum of squares) is done with explicitly rounded FP64 operations in the same
// order as the definition, so distances and the ordering are reproducible.
template <int D>
__device__ inline void mi_exact(const double* H, double* d) {
#pragma unroll
  for (int c = D - 1; c >= 0; c--) {
    double n = rint(__ddiv_rn(d[c], H[c * D + c]));
#pragma unroll
    for (int a = 0; a <= c; a++) d[a] = __dsub_rn(d[a], __dmul_rn(n, H[a * D + c]));
  }
}

template <int D, int NB>
__global__ void k_knn_features(FeatArgs a) {
  const int il = blockIdx.x * blockDim.x + threadIdx.x;
  const RepGeom& g = a.geom[a.rep];
  if (il >= g.n) return;
  const int64_t N = a.ntot;
  const int64_t gi = g.off + il;
  double H[9];
  for (int k = 0; k < 9; k++) H[k] = g.H[k];
  H[1] = a.tilt;
  const int ci = a.cell[gi];
  int cc[3] = {ci % g.nc[0], (ci / g.nc[0]) % g.nc[1], D == 3 ? ci / (g.nc[0] * g.nc[1]) : 0};
  double xi[3];
  for (int c = 0; c < D; c++) xi[c] = a.x[c * N + gi];
  // best NB candidates, sorted ascending by (s, caller index)
  double bs[NB];
  int bj[NB];
  for (int k = 0; k < NB; k++) {
    bs[k] = INFINITY;
    bj[k] = 0x7fffffff;
  }
  const int h = a.half;  // stencil half-width in cells
  const int zh = D == 3 ? h : 0;
  for (int dz = -zh; dz <= zh; dz++)
    for (int dy = -h; dy <= h; dy++)
      for (int dx = -h; dx <= h; dx++) {
        int nx = ((cc[0] + dx) % g.nc[0] + g.nc[0]) % g.nc[0];
        int ny = ((cc[1] + dy) % g.nc[1] + g.nc[1]) % g.nc[1];
        int nz = D == 3 ? ((cc[2] + dz) % g.nc[2] + g.nc[2]) % g.nc[2] : 0;
        int cj = nx + g.nc[0] * (ny + g.nc[1] * nz);
        // stencils that wrap onto the same cell twice are visited once
        bool dup = false;
        for (int ez = -zh; ez <= dz && !dup; ez++)
          for (int ey = -h; ey <= h && !dup; ey++)
            for (int ex = -h; ex <= h; ex++) {
              if (ez == dz && ey == dy && ex == dx) goto done_dup;
              {
                int mx = ((cc[0] + ex) % g.nc[0] + g.nc[0]) % g.nc[0];
                int my = ((cc[1] + ey) % g.nc[1] + g.nc[1]) % g.nc[1];
                int mz = D == 3 ? ((cc[2] + ez) % g.nc[2] + g.nc[2]) % g.nc[2] : 0;
                if (mx + g.nc[0] * (my + g.nc[1] * mz) == cj) {
                  dup = true;
                  break;
                }
              }
            }
      done_dup:
        if (dup) continue;
        for (int jl = a.cstart[g.cell_off + cj]; jl < a.cstart[g.cell_off + cj + 1]; jl++) {
          if (jl == il) continue;
          const int64_t gj = g.off + jl;
          double d[3];
          for (int c = 0; c < D; c++) d[c] = __dsub_rn(a.x[c * N + gj], xi[c]);
          mi_exact<D>(H, d);
          double s = __dmul_rn(d[0], d[0]);
          for (int c = 1; c < D; c++) s = __dadd_rn(s, __dmul_rn(d[c], d[c]));
          const int uj = a.perm[gj];
          if (s > bs[NB - 1] || (s == bs[NB - 1] && uj > bj[NB - 1])) continue;
          int k = NB - 1;
          while (k > 0 && (bs[k - 1] > s || (bs[k - 1] == s && bj[k - 1] > uj))) {
            bs[k] = bs[k - 1];
            bj[k] = bj[k - 1];
            k--;
          }
          bs[k] = s;
          bj[k] = uj;
        }
      }
  // the stencil reaches at least half * (smallest cell width); beyond that a
  // nearer atom could have been missed
  if (!(bs[NB - 1] < a.reach2)) atomicExch(a.err, 1);
  const int64_t row = a.row0 + a.perm[gi];  // caller order
  for (int k = 0; k < NB; k++) {
    const int64_t gj = g.off + a.inv[g.off + bj[k]];
    double d[3];
    for (int c = 0; c < D; c++) d[c] = __dsub_rn(a.x[c * N + gj], xi[c]);
    mi_exact<D>(H, d);
    for (int c = 0; c < D; c++) {
      if (a.f64) a.f64[row * a.width64 + k * D + c] = d[c];
      a.bf[row * a.width + k * D + c] = __float2bfloat16_rn((float)d[c]);
    }
  }
  const int ty = a.type[gi];
  for (int t = 0; t < a.n_types; t++) {
    double v = t == ty ? 1.0 : 0.0;
    if (a.f64) a.f64[row * a.width64 + NB * D + t] = v;
    a.bf[row * a.width + NB * D + t] = __float2bfloat16_rn((float)v);
  }
  for (int k = NB * D + a.n_types; k < a.width; k++) a.bf[row * a.width + k] = __float2bfloat16_rn(0.f);
}

cudaError_t launch_knn_features(int dim, const FeatArgs& a, int n, cudaStream_t s) {
  count_launch();
  if (a.nb != 32) return cudaErrorInvalidValue;
  if (dim == 2) k_knn_features<2, 32><<<(n + 63) / 64, 64, 0, s>>>(a);
  else k_knn_features<3, 32><<<(n + 63) / 64, 64, 0, s>>>(a);
  return cudaGetLastError();
}

// Non-affine displacement per unit strain of every atom of a replica after a
// step, in caller order: u = mi(x - x_start) / dgamma (FP64 difference, FP32
// result), the training target of the warm start.
template <int D>
__global__ void k_step_target(const double* x, const double* xs, int64_t N, int64_t off, int n,
                              const int32_t* perm, const double* Hd, double inv_dg, float* out) {
  int il = blockIdx.x * blockDim.x + threadIdx.x;
  if (il >= n) return;
  int64_t gi = off + il;
  double H[9];
  for (int k = 0; k < 9; k++) H[k] = Hd[k];
  double d[3];
  for (int c = 0; c < D; c++) d[c] = x[c * N + gi] - xs[c * N + gi];
  min_image<D>(H, d);
  const int u = perm[gi];
  for (int c = 0; c < D; c++) out[(int64_t)u * D + c] = (float)(d[c] * inv_dg);
}

cudaError_t launch_step_target(int dim, const double* x, const double* xs, int64_t N, int64_t off,
                               int n, const int32_t* perm, const double* H, double inv_dg,
                               float* out, cudaStream_t s) {
  count_launch();
  if (dim == 2) k_step_target<2><<<(n + 127) / 128, 128, 0, s>>>(x, xs, N, off, n, perm, H, inv_dg, out);
  else k_step_target<3><<<(n + 127) / 128, 128, 0, s>>>(x, xs, N, off, n, perm, H, inv_dg, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- MLP
// m16n8k16 BF16 MMA, FP32 accumulate (PTX ISA operand layouts):
//   A 16x16 row-major: a[0..1] (g, 2t..2t+1), a[2..3] (g+8, 2t..), a[4..5] (g, 2t+8..), a[6..7] (g+8, 2t+8..)
//   B 16x8 col-major:  b[0..1] (k = 2t..2t+1, n = g), b[2..3] (k = 2t+8.., n = g)
//   C 16x8:            c[0..1] (g, 2t..2t+1), c[2..3] (g+8, 2t..2t+1)
// with g = lane / 4, t = lane % 4.
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment loads for mma.m16n8k16 from shared memory (rows of 8 BF16 at
// 16-byte aligned addresses, one address per lane): x4 gives an A fragment
// (16 rows x 16 k), x2 a B fragment from 8 rows of W (n) with k contiguous,
// x2.trans a B fragment from 16 rows of a k-major matrix (k rows, n contiguous).
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// Layer l of the forward pass for one warp's 16 rows: Z = A W^T + b, A is
// [16 x K] (row stride lda, BF16) in shared memory, W is [NOUT x K] BF16
// (row stride ldw) in shared memory; the 16 x NOUT result is written to the
// FP32 array z (row stride ldz).
template <int K, int NOUT>
__device__ __forceinline__ void warp_layer(const __nv_bfloat16* A, int lda, const __nv_bfloat16* W,
                                           int ldw, const float* bias, float* z, int ldz) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  const int brow = lane & 7, bcol = ((lane >> 3) & 1) * 8;
#pragma unroll
  for (int nt = 0; nt < NOUT / 8; nt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < K / 16; kt++) {
      const int k0 = kt * 16;
      uint32_t a[4], b[2];
      ldsm_x4(a, A + arow * lda + k0 + acol);
      ldsm_x2(b, W + (nt * 8 + brow) * ldw + k0 + bcol);
      mma16816(c, a, b);
    }
    const int col = nt * 8 + 2 * t;
    z[g * ldz + col] = c[0] + bias[col];
    z[g * ldz + col + 1] = c[1] + bias[col + 1];
    z[(g + 8) * ldz + col] = c[2] + bias[col];
    z[(g + 8) * ldz + col + 1] = c[3] + bias[col + 1];
  }
}

// Shared-memory plan of the MLP kernels (sizes in elements).
constexpr int kRows = 32;   // rows per CTA tile (2 warps x 16)
constexpr int kThreads = 64;
struct MlpSmem {
  static constexpr int w1 = kHid * kIn, w2 = kHid * kHid, w3 = kHid * kHid, w4 = kOutPad * kHid;
};

__device__ void load_weights(const MlpDev& m, __nv_bfloat16* sw, float* sb) {
  const int nw = MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3 + MlpSmem::w4;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) sw[k] = m.wbf[k];
  for (int k = threadIdx.x; k < 3 * kHid + kOutPad; k += blockDim.x) sb[k] = m.b[k];
}

// Forward for rows [row0, row0 + 64): keeps Z of every layer (FP32) and the
// BF16 activations in shared memory; returns Y in zo (rows x kOutPad).
__device__ void mlp_forward_tile(const __nv_bfloat16* sw, const float* sb, const __nv_bfloat16* X,
                                 int64_t rows, int64_t row0, __nv_bfloat16* sx, __nv_bfloat16* sa,
                                 float* sz, float* zo) {
  const int warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kRows * kIn; k += blockDim.x) {
    int64_t r = row0 + k / kIn;
    sx[k] = r < rows ? X[r * kIn + (k % kIn)] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  const __nv_bfloat16* W1 = sw;
  const __nv_bfloat16* W2 = W1 + MlpSmem::w1;
  const __nv_bfloat16* W3 = W2 + MlpSmem::w2;
  const __nv_bfloat16* W4 = W3 + MlpSmem::w3;
  const int r0 = warp * 16;
  // layer 1..3 with GELU; Z_l kept in sz[l]
  const __nv_bfloat16* Ain = sx + r0 * kIn;
  int lda = kIn;
  for (int l = 0; l < 3; l++) {
    float* z = sz + l * kRows * kHid + r0 * kHid;
    if (l == 0) warp_layer<kIn, kHid>(Ain, lda, W1, kIn, sb, z, kHid);
    else warp_layer<kHid, kHid>(Ain, lda, l == 1 ? W2 : W3, kHid, sb + l * kHid, z, kHid);
    __syncwarp();
    __nv_bfloat16* a = sa + l * kRows * kHid + r0 * kHid;
    for (int k = threadIdx.x & 31; k < 16 * kHid; k += 32) a[k] = __float2bfloat16_rn(gelu(z[k]));
    __syncwarp();
    Ain = a;
    lda = kHid;
  }
  warp_layer<kHid, kOutPad>(Ain, kHid, W4, kHid, sb + 3 * kHid, zo + r0 * kOutPad, kOutPad);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Inference (forward only).  Every warp carries 16-row tiles through the four
// layers on its own; the weights are staged once per CTA in shared memory
// with padded rows (88 or 136 BF16 = 176 or 272 bytes, so eight consecutive
// rows start in different banks and ldmatrix reads them without conflicts).
// A layer's 16 x NOUT result stays in the MMA accumulators until bias and
// GELU are applied and it is written, as BF16, over the warp's activation
// tile.  Arithmetic and accumulation order are those of mlp_forward_tile.
constexpr int kInferWarps = 16;
constexpr int kLdIn = kIn + 8;
constexpr int kLdHid = kHid + 8;


// acc[nt] = A (16 x K, BF16, row stride lda) times W^T (W: NOUT x K, row
// stride ldw), FP32 accumulators in the mma.m16n8k16 layout
template <int K, int NOUT>
__device__ __forceinline__ void warp_mma_layer(const __nv_bfloat16* A, int lda,
                                               const __nv_bfloat16* W, int ldw, float (*acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  const int brow = lane & 7, bcol = ((lane >> 3) & 1) * 8;
#pragma unroll
  for (int nt = 0; nt < NOUT / 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
  for (int kt = 0; kt < K / 16; kt++) {
    uint32_t a[4];
    ldsm_x4(a, A + arow * lda + kt * 16 + acol);
#pragma unroll
    for (int nt = 0; nt < NOUT / 8; nt++) {
      uint32_t b[2];
      ldsm_x2(b, W + (nt * 8 + brow) * ldw + kt * 16 + bcol);
      mma16816(acc[nt], a, b);
    }
  }
}

// out (16 x NOUT, BF16, row stride ldo) = GELU(acc + bias)
template <int NOUT>
__device__ __forceinline__ void store_gelu(float (*acc)[4], const float* bias, __nv_bfloat16* out,
                                           int ldo) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NOUT / 8; nt++) {
    const int col = nt * 8 + 2 * t;
    const float b0 = bias[col], b1 = bias[col + 1];
    *reinterpret_cast<uint32_t*>(out + g * ldo + col) =
        pack2(__float2bfloat16_rn(gelu(acc[nt][0] + b0)), __float2bfloat16_rn(gelu(acc[nt][1] + b1)));
    *reinterpret_cast<uint32_t*>(out + (g + 8) * ldo + col) =
        pack2(__float2bfloat16_rn(gelu(acc[nt][2] + b0)), __float2bfloat16_rn(gelu(acc[nt][3] + b1)));
  }
}

__global__ void __launch_bounds__(kInferWarps * 32, 1)
    k_mlp_infer(MlpDev m, const __nv_bfloat16* X, int64_t rows, float* Y, int nout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(smraw);  // [kHid][kLdIn]
  __nv_bfloat16* w2 = w1 + kHid * kLdIn;                          // [kHid][kLdHid]
  __nv_bfloat16* w3 = w2 + kHid * kLdHid;                         // [kHid][kLdHid]
  __nv_bfloat16* w4 = w3 + kHid * kLdHid;                         // [kOutPad][kLdHid]
  float* sb = reinterpret_cast<float*>(w4 + kOutPad * kLdHid);    // [3 kHid + kOutPad]
  __nv_bfloat16* tiles = reinterpret_cast<__nv_bfloat16*>(sb + 3 * kHid + kOutPad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* xs = tiles + warp * 16 * (kLdIn + kLdHid);  // [16][kLdIn]
  __nv_bfloat16* act = xs + 16 * kLdIn;                       // [16][kLdHid]
  const __nv_bfloat16* g1 = m.wbf;
  const __nv_bfloat16* g2 = g1 + kHid * kIn;
  const __nv_bfloat16* g3 = g2 + kHid * kHid;
  const __nv_bfloat16* g4 = g3 + kHid * kHid;
  for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x) w1[(k / kIn) * kLdIn + k % kIn] = g1[k];
  for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) {
    w2[(k / kHid) * kLdHid + k % kHid] = g2[k];
    w3[(k / kHid) * kLdHid + k % kHid] = g3[k];
  }
  for (int k = threadIdx.x; k < kOutPad * kHid; k += blockDim.x)
    w4[(k / kHid) * kLdHid + k % kHid] = g4[k];
  for (int k = threadIdx.x; k < 3 * kHid + kOutPad; k += blockDim.x) sb[k] = m.b[k];
  __syncthreads();
  float acc[kHid / 8][4];
  const int64_t ntiles = (rows + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * kInferWarps + warp; tile < ntiles;
       tile += (int64_t)gridDim.x * kInferWarps) {
    const int64_t r0 = tile * 16;
    // the tile's 16 input rows, 16-byte words (X rows are 160 bytes)
    for (int w = lane; w < 16 * (kIn / 8); w += 32) {
      const int r = w / (kIn / 8), c = w % (kIn / 8);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + r < rows) v = *reinterpret_cast<const uint4*>(X + (r0 + r) * kIn + c * 8);
      *reinterpret_cast<uint4*>(xs + r * kLdIn + c * 8) = v;
    }
    __syncwarp();
    warp_mma_layer<kIn, kHid>(xs, kLdIn, w1, kLdIn, acc);
    store_gelu<kHid>(acc, sb, act, kLdHid);
    __syncwarp();
    warp_mma_layer<kHid, kHid>(act, kLdHid, w2, kLdHid, acc);
    __syncwarp();  // every lane has read the tile before it is overwritten
    store_gelu<kHid>(acc, sb + kHid, act, kLdHid);
    __syncwarp();
    warp_mma_layer<kHid, kHid>(act, kLdHid, w3, kLdHid, acc);
    __syncwarp();
    store_gelu<kHid>(acc, sb + 2 * kHid, act, kLdHid);
    __syncwarp();
    float y[kOutPad / 8][4];
    warp_mma_layer<kHid, kOutPad>(act, kLdHid, w4, kLdHid, y);
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < kOutPad / 8; nt++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int col = nt * 8 + 2 * t + e;
        if (col >= nout) continue;
        const float bo = sb[3 * kHid + col];
        if (r0 + g < rows) Y[(r0 + g) * nout + col] = y[nt][e] + bo;
        if (r0 + g + 8 < rows) Y[(r0 + g + 8) * nout + col] = y[nt][2 + e] + bo;
      }
    __syncwarp();  // the tile buffers are free for the next tile
  }
}

// Fused forward + backward of the loss 0.5/m sum (Y - T)^2 for rows
// [row0, row0 + 64) of the CTA's share; each CTA accumulates its weight and
// bias gradients in FP32 shared memory and writes them to its own partial
// slot (summed afterwards in CTA order: deterministic).
//
// Backward per layer l (Z_l = A_{l-1} W_l^T + b_l):
//   dW_l = dZ_l^T A_{l-1},  db_l = sum_rows dZ_l,  dA_{l-1} = dZ_l W_l,
//   dZ_{l-1} = dA_{l-1} * GELU'(Z_{l-1}).
// dW uses the tensor cores with the rows as the reduction dimension.
__device__ __forceinline__ void dw_accumulate(const __nv_bfloat16* dZt, int ldd, int nout,
                                              const __nv_bfloat16* At, int lda, int nin,
                                              float* gw) {
  // gw[o][i] += sum_r dZ[r][o] A[r][i]; dZt is dZ transposed [nout x 64],
  // At is A transposed [nin x 64], both BF16 with the row dimension contiguous.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ntile_o = nout / 16, ntile_i = nin / 8;
  const int nwarps = blockDim.x >> 5;
  for (int tile = warp; tile < ntile_o * ntile_i; tile += nwarps) {
    const int ot = tile / ntile_i, it = tile % ntile_i;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < kRows / 16; kt++) {
      const int k0 = kt * 16;
      uint32_t a[4], b[2];
      const __nv_bfloat16* ar0 = dZt + (ot * 16 + g) * ldd + k0;
      const __nv_bfloat16* ar1 = dZt + (ot * 16 + g + 8) * ldd + k0;
      a[0] = pack2(ar0[2 * t], ar0[2 * t + 1]);
      a[1] = pack2(ar1[2 * t], ar1[2 * t + 1]);
      a[2] = pack2(ar0[2 * t + 8], ar0[2 * t + 9]);
      a[3] = pack2(ar1[2 * t + 8], ar1[2 * t + 9]);
      const __nv_bfloat16* br = At + (it * 8 + g) * lda + k0;
      b[0] = pack2(br[2 * t], br[2 * t + 1]);
      b[1] = pack2(br[2 * t + 8], br[2 * t + 9]);
      mma16816(c, a, b);
    }
    const int o0 = ot * 16 + g, i0 = it * 8 + 2 * t;
    gw[o0 * nin + i0] += c[0];
    gw[o0 * nin + i0 + 1] += c[1];
    gw[(o0 + 8) * nin + i0] += c[2];
    gw[(o0 + 8) * nin + i0 + 1] += c[3];
  }
}

__global__ void __launch_bounds__(kThreads) k_mlp_grad(MlpDev m, const __nv_bfloat16* X, const float* T,
                                                  int64_t rows, int nout, float* partial,
                                                  float* loss_partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* sx = sw + MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3 + MlpSmem::w4;
  __nv_bfloat16* sa = sx + kRows * kIn;
  float* sb = reinterpret_cast<float*>(sa + 3 * kRows * kHid);
  float* sz = sb + 3 * kHid + kOutPad;
  float* zo = sz + 3 * kRows * kHid;
  __nv_bfloat16* dzt = reinterpret_cast<__nv_bfloat16*>(zo + kRows * kOutPad);  // [kHid][kRows]
  __nv_bfloat16* at = dzt + kHid * kRows;                                       // [kHid][kRows]
  float* dz = reinterpret_cast<float*>(at + kHid * kRows);                      // [kRows][kHid]
  float* gacc = m.gscratch + (int64_t)blockIdx.x * kNumParams;                  // this CTA's sums
  load_weights(m, sw, sb);
  for (int k = threadIdx.x; k < kNumParams; k += blockDim.x) gacc[k] = 0.f;
  __syncthreads();
  const __nv_bfloat16* W[4] = {sw, sw + MlpSmem::w1, sw + MlpSmem::w1 + MlpSmem::w2,
                               sw + MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3};
  const int woff[4] = {0, MlpSmem::w1, MlpSmem::w1 + MlpSmem::w2,
                       MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3};
  const int boff = MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3 + MlpSmem::w4;
  const int nin_l[4] = {kIn, kHid, kHid, kHid};
  const int nout_l[4] = {kHid, kHid, kHid, kOutPad};
  float lsum = 0.f;
  const float inv_m = 1.0f / (float)rows;
  for (int64_t row0 = (int64_t)blockIdx.x * kRows; row0 < rows; row0 += (int64_t)gridDim.x * kRows) {
    mlp_forward_tile(sw, sb, X, rows, row0, sx, sa, sz, zo);
    // dY = (Y - T) / m on the valid rows and outputs (padding columns zero)
    for (int k = threadIdx.x; k < kRows * kOutPad; k += blockDim.x) {
      const int r = k / kOutPad, o = k % kOutPad;
      const int64_t gr = row0 + r;
      float d = 0.f;
      if (gr < rows && o < nout) {
        float e = zo[k] - T[gr * nout + o];
        lsum += 0.5f * e * e;
        d = e * inv_m;
      }
      dz[r * kHid + o] = d;  // dZ of the output layer (linear), width kOutPad
    }
    __syncthreads();
    for (int l = 3; l >= 0; l--) {
      const int nin = nin_l[l], no = nout_l[l];
      const __nv_bfloat16* Aprev = l == 0 ? sx : sa + (l - 1) * kRows * kHid;
      const int ldprev = l == 0 ? kIn : kHid;
      // transposed BF16 copies of dZ_l and A_{l-1} for the dW tensor-core product
      for (int k = threadIdx.x; k < no * kRows; k += blockDim.x) {
        const int o = k / kRows, r = k % kRows;
        dzt[o * kRows + r] = __float2bfloat16_rn(dz[r * kHid + o]);
      }
      for (int k = threadIdx.x; k < nin * kRows; k += blockDim.x) {
        const int i = k / kRows, r = k % kRows;
        at[i * kRows + r] = Aprev[r * ldprev + i];
      }
      __syncthreads();
      dw_accumulate(dzt, kRows, no, at, kRows, nin, gacc + woff[l]);
      for (int o = threadIdx.x; o < no; o += blockDim.x) {
        float sbias = 0.f;
        for (int r = 0; r < kRows; r++) sbias += dz[r * kHid + o];
        gacc[boff + (l == 3 ? 3 * kHid : l * kHid) + o] += sbias;
      }
      __syncthreads();
      if (l > 0) {
        // dA_{l-1}[r][i] = sum_o dZ[r][o] W_l[o][i] on the tensor cores (dZ
        // in BF16, as for dW; FP32 accumulation), then times GELU'(Z_{l-1}).
        // dZ goes row-major into the transposed-A buffer, free after dW.
        const __nv_bfloat16* Wl = W[l];
        float* zprev = sz + (l - 1) * kRows * kHid;
        __nv_bfloat16* dzr = at;  // [kRows][no]
        for (int k = threadIdx.x; k < kRows * no; k += blockDim.x)
          dzr[k] = __float2bfloat16_rn(dz[(k / no) * kHid + k % no]);
        __syncthreads();
        {
          const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
          const int r0 = warp * 16;
          const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
          const int krow = (lane & 7) + ((lane >> 3) & 1) * 8;
          for (int nt = 0; nt < nin / 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            for (int kt = 0; kt < no / 16; kt++) {
              uint32_t a[4], b[2];
              ldsm_x4(a, dzr + (r0 + arow) * no + kt * 16 + acol);
              ldsm_x2_trans(b, Wl + (kt * 16 + krow) * nin + nt * 8);
              mma16816(c, a, b);
            }
            const int i0 = nt * 8 + 2 * t;
            float* z0 = zprev + (r0 + g) * kHid + i0;
            float* z1 = zprev + (r0 + g + 8) * kHid + i0;
            z0[0] = c[0] * gelu_grad(z0[0]);
            z0[1] = c[1] * gelu_grad(z0[1]);
            z1[0] = c[2] * gelu_grad(z1[0]);
            z1[1] = c[3] * gelu_grad(z1[1]);
          }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kRows * kHid; k += blockDim.x)
          dz[k] = sz[(l - 1) * kRows * kHid + k];
        __syncthreads();
      }
    }
  }
  // loss partial
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  __shared__ float ls[kThreads / 32];
  if ((threadIdx.x & 31) == 0) ls[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kThreads / 32; w++) t += ls[w];
    loss_partial[blockIdx.x] = t * inv_m;
  }
  (void)partial;
}

// Sum the per-CTA gradients in CTA order, then AdamW with FP32 master weights.
__global__ void k_mlp_reduce(MlpDev m, int nblocks, float* grad_out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNumParams) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; b++) s += m.gscratch[(int64_t)b * kNumParams + k];
  grad_out[k] = s;
}

__global__ void k_mlp_adamw(MlpDev m, const float* grad, float lr, float beta1, float beta2,
                            float eps, float wd, float bc1, float bc2) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNumParams) return;
  const bool is_w = k < kNumWeights;
  float gk = grad[k];
  float mk = beta1 * m.m1[k] + (1.f - beta1) * gk;
  float vk = beta2 * m.m2[k] + (1.f - beta2) * gk * gk;
  m.m1[k] = mk;
  m.m2[k] = vk;
  float p = m.master[k];
  if (is_w) p -= lr * wd * p;
  p -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  // padded rows/columns stay zero
  if (!m.mask[k]) p = 0.f;
  m.master[k] = p;
  if (is_w) m.wbf[k] = __float2bfloat16_rn(p);
  else m.b[k - kNumWeights] = p;
}

size_t mlp_smem_forward() {
  return sizeof(__nv_bfloat16) * (MlpSmem::w1 + MlpSmem::w2 + MlpSmem::w3 + MlpSmem::w4 +
                                  kRows * kIn + 3 * kRows * kHid) +
         sizeof(float) * (3 * kHid + kOutPad + 3 * kRows * kHid + kRows * kOutPad);
}

size_t mlp_smem_grad() {
  return mlp_smem_forward() + sizeof(__nv_bfloat16) * (2 * kHid * kRows) +
         sizeof(float) * (kRows * kHid);
}

cudaError_t launch_mlp_forward(const MlpDev& m, const __nv_bfloat16* X, int64_t rows, float* Y,
                               int nout, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0u || nout > kOutPad) return cudaErrorInvalidValue;
  const size_t smem = sizeof(__nv_bfloat16) * (kHid * kLdIn + 2 * kHid * kLdHid + kOutPad * kLdHid +
                                               kInferWarps * 16 * (kLdIn + kLdHid)) +
                      sizeof(float) * (3 * kHid + kOutPad);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (rows + 15) / 16;
  int blocks = (int)std::min<int64_t>((ntiles + kInferWarps - 1) / kInferWarps, sm_count());
  if (blocks < 1) blocks = 1;
  count_launch();
  k_mlp_infer<<<blocks, kInferWarps * 32, smem, s>>>(m, X, rows, Y, nout);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const MlpDev& m, const __nv_bfloat16* X, const float* T, int64_t rows,
                            int nout, int blocks, float* grad_out, float* loss_partial,
                            cudaStream_t s) {
  size_t smem = mlp_smem_grad();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  k_mlp_grad<<<blocks, kThreads, smem, s>>>(m, X, T, rows, nout, nullptr, loss_partial);
  count_launch();
  k_mlp_reduce<<<(kNumParams + 255) / 256, 256, 0, s>>>(m, blocks, grad_out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adamw(const MlpDev& m, const float* grad, float lr, float beta1, float beta2,
                             float eps, float wd, float bc1, float bc2, cudaStream_t s) {
  count_launch();
  k_mlp_adamw<<<(kNumParams + 255) / 256, 256, 0, s>>>(m, grad, lr, beta1, beta2, eps, wd, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace aqs
