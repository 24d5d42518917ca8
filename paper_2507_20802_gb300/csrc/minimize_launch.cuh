// minimize_launch.cuh -- launch helpers of the minimiser instantiations.
#pragma once
#include "minimize_kernel.cuh"

namespace aqs {

inline size_t smem_fixed(int nt) {
  return sizeof(double) * (kNumRed * 33 + 27 * 3) + sizeof(float) * (27 * 3 + 3) +
         sizeof(float) * kOffLane + sizeof(PairCoef) * nt * nt + 64;
}

inline size_t pub_size(int dim) { return dim == 2 ? sizeof(Pub<2>) : sizeof(Pub<3>); }

inline size_t minimize_smem_bytes_impl(int dim, int npc, int nrep, int nt, int cap, int mem) {
  // records: the whole replica (mode 2), the CTA's own atoms (modes 1, 3), or
  // none (mode 0 keeps them in the global record array)
  size_t pub = pub_size(dim) * (size_t)(mem == 2 ? nrep : (mem == 0 ? 0 : npc));
  return pub + smem_fixed(nt) + (mem >= 1 ? sizeof(uint32_t) * (size_t)cap * npc : 0);
}

constexpr size_t kSmemLimit = 220 * 1024;

inline int choose_mem(int dim, int npc, int nrep, int nt, int cap, int want = -1) {
  if (want >= 0 && want < kNumStaging &&
      minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, want) <= kSmemLimit)
    return want;
  if (minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, 2) <= kSmemLimit) return 2;
  if (minimize_smem_bytes_impl(dim, npc, nrep, nt, cap, 1) <= kSmemLimit) return 1;
  return 0;
}

// threads per atom of the force phase a launch can use: `want` (2) when
// npc * want threads fit in one CTA, else 1
inline int effective_tpa(int npc, int want) { return (want == 2 && npc * 2 <= 1024) ? 2 : 1; }

inline void choose_apt(int dim, int npc, int* apt, int* threads, int tpa = 1) {
  if (tpa > 1) {
    *apt = 1;
    *threads = ((npc * tpa + 31) / 32) * 32;
    return;
  }
  *apt = npc <= 512 ? 1 : (npc <= 1024 ? 2 : (npc <= 2048 ? 4 : 8));
  // lean launches hold little per-thread state and may use up to 1024
  // threads: halve the atoms per thread where the result is still lean
  if (minimize_is_lean(dim, *apt) && minimize_is_lean(dim, *apt / 2)) *apt /= 2;
  int t = (npc + *apt - 1) / *apt;
  *threads = ((t + 31) / 32) * 32;
}

template <int D, bool MIXED, int APT, int MEM, int TPA, bool GB>
cudaError_t run_t(const MinArgs* a, int n_clusters, int C, int threads, size_t smem,
                         cudaStream_t s, int* max_clusters) {
  auto kern = k_minimize<D, MIXED, APT, MEM, TPA, GB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (MEM == 0) {  // little shared memory: leave the rest of the SM's array to L1
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxL1);
    if (e != cudaSuccess) return e;
  }
  if constexpr (GB) {
    // cooperative launch of n_clusters replicas x C consecutive CTAs; every CTA
    // must be resident (the launch fails otherwise, it never waits)
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (max_clusters) {
      *max_clusters = per_sm * sm_count() / C;
      return cudaSuccess;
    }
    if ((int64_t)n_clusters * C > (int64_t)per_sm * sm_count()) return cudaErrorCooperativeLaunchTooLarge;
    MinArgs args = *a;
    args.gb_C = C;
    void* params[] = {&args};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(n_clusters * C), dim3(threads),
                                       params, smem, s);
  }
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(n_clusters * C);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, *a);
}

template <int D, bool MIXED, int MEM, int TPA, bool GB>
cudaError_t run_apt(const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                           cudaStream_t s, int* max_clusters) {
  int apt, threads;
  choose_apt(D, npc, &apt, &threads, TPA);
  if (threads > ((minimize_is_lean(D, apt) || TPA > 1) ? 1024 : 512)) return cudaErrorInvalidValue;
  if constexpr (TPA > 1) {
    return run_t<D, MIXED, 1, MEM, TPA, GB>(a, n_clusters, C, threads, smem, s, max_clusters);
  } else {
    switch (apt) {
      case 1: return run_t<D, MIXED, 1, MEM, 1, GB>(a, n_clusters, C, threads, smem, s, max_clusters);
      case 2: return run_t<D, MIXED, 2, MEM, 1, GB>(a, n_clusters, C, threads, smem, s, max_clusters);
      case 4: return run_t<D, MIXED, 4, MEM, 1, GB>(a, n_clusters, C, threads, smem, s, max_clusters);
      default: return run_t<D, MIXED, 8, MEM, 1, GB>(a, n_clusters, C, threads, smem, s, max_clusters);
    }
  }
}

template <int D, bool MIXED, int TPA, bool GB = false>
cudaError_t run_mem(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                           cudaStream_t s, int* max_clusters) {
  if constexpr (GB) {  // global neighbour records only
    if (mem == 0) return run_apt<D, MIXED, 0, TPA, true>(a, n_clusters, C, npc, smem, s, max_clusters);
    return run_apt<D, MIXED, 3, TPA, true>(a, n_clusters, C, npc, smem, s, max_clusters);
  } else {
    switch (mem) {
      case 3: return run_apt<D, MIXED, 3, TPA, false>(a, n_clusters, C, npc, smem, s, max_clusters);
      case 2: return run_apt<D, MIXED, 2, TPA, false>(a, n_clusters, C, npc, smem, s, max_clusters);
      case 1: return run_apt<D, MIXED, 1, TPA, false>(a, n_clusters, C, npc, smem, s, max_clusters);
      default: return run_apt<D, MIXED, 0, TPA, false>(a, n_clusters, C, npc, smem, s, max_clusters);
    }
  }
}

// one instantiation unit per (dimension, precision)
cudaError_t run_mem_2_fp64(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                           cudaStream_t s, int* max_clusters);
cudaError_t run_mem_2_mixed(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                            cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_fp64(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                           cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_mixed(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                            cudaStream_t s, int* max_clusters);
// grid-barrier (cooperative) launches, one unit each
cudaError_t run_mem_2_fp64_gb(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                              size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_2_mixed_gb(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                               size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_fp64_gb(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                              size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_mixed_gb(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                               size_t smem, cudaStream_t s, int* max_clusters);
// the split force phase (two threads per atom), one unit each
cudaError_t run_mem_2_fp64_t2(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                              size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_2_mixed_t2(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                               size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_fp64_t2(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                              size_t smem, cudaStream_t s, int* max_clusters);
cudaError_t run_mem_3_mixed_t2(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                               size_t smem, cudaStream_t s, int* max_clusters);

}  // namespace aqs
