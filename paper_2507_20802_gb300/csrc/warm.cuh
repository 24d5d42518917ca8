// warm.cuh -- learned warm start: feature and MLP launchers (2D workloads).
#pragma once
#include <cuda_bf16.h>

#include "aqs_internal.cuh"

namespace aqs {

constexpr int kNb = 32;        // nearest neighbours per atom
constexpr int kFeat2D = kNb * 2 + 2;  // 2D displacements + species one-hot
constexpr int kIn = 80;        // input width padded to a multiple of 16
constexpr int kHid = 128;      // hidden width
constexpr int kOutPad = 16;    // output rows of the last layer padded for the MMA tile
constexpr int kNumWeights = kHid * kIn + 2 * kHid * kHid + kOutPad * kHid;
constexpr int kNumBiases = 3 * kHid + kOutPad;
constexpr int kNumParams = kNumWeights + kNumBiases;

// parameters: [W1 (kHid x kIn), W2, W3 (kHid x kHid), W4 (kOutPad x kHid), b1, b2, b3, b4]
struct MlpDev {
  __nv_bfloat16* wbf;  // BF16 weights used by the tensor cores [kNumWeights]
  float* b;            // biases [kNumBiases]
  float* master;       // FP32 master copy of all parameters [kNumParams]
  float* m1;           // AdamW first moments
  float* m2;           // AdamW second moments
  const uint8_t* mask; // 1 where a parameter is real (0 in the padding)
  float* gscratch;     // per-CTA gradient sums [blocks][kNumParams]
};

struct FeatArgs {
  const RepGeom* geom;
  int rep;
  double tilt;         // current H[0][1] of the replica
  const double* x;
  const int32_t* type, *cell, *cstart, *perm, *inv;
  int64_t ntot;
  int nb, n_types, half;
  double reach2;       // (half * smallest cell width)^2: the stencil is exact below it
  __nv_bfloat16* bf;   // [rows][width] BF16 features
  int width;
  double* f64;         // [rows][width64] FP64 features (nullable)
  int width64;
  int64_t row0;        // first output row
  int* err;            // set to 1 if the stencil could have missed a neighbour
};

cudaError_t launch_knn_features(int dim, const FeatArgs& a, int n, cudaStream_t s);
cudaError_t launch_step_target(int dim, const double* x, const double* xs, int64_t N, int64_t off,
                               int n, const int32_t* perm, const double* H, double inv_dg,
                               float* out, cudaStream_t s);
size_t mlp_smem_forward();
size_t mlp_smem_grad();
cudaError_t launch_mlp_forward(const MlpDev& m, const __nv_bfloat16* X, int64_t rows, float* Y,
                               int nout, cudaStream_t s);
cudaError_t launch_mlp_grad(const MlpDev& m, const __nv_bfloat16* X, const float* T, int64_t rows,
                            int nout, int blocks, float* grad_out, float* loss_partial,
                            cudaStream_t s);
cudaError_t launch_mlp_adamw(const MlpDev& m, const float* grad, float lr, float beta1, float beta2,
                             float eps, float wd, float bc1, float bc2, cudaStream_t s);

}  // namespace aqs
