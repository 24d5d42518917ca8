// minimize_2d_fp64_t2.cu -- instantiation of the persistent minimiser for
// dimension 2, FP64 precision, with the split force phase (two threads per
// atom); its own unit so that the variants compile in parallel.
#include "minimize_launch.cuh"

namespace aqs {

cudaError_t run_mem_2_fp64_t2(int mem, const MinArgs* a, int n_clusters, int C, int npc, size_t smem,
                  cudaStream_t s, int* max_clusters) {
  return run_mem<2, false, 2>(mem, a, n_clusters, C, npc, smem, s, max_clusters);
}

}  // namespace aqs
