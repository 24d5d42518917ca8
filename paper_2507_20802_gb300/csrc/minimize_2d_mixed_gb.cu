// minimize_2d_mixed_gb.cu -- instantiation of the persistent minimiser for
// dimension 2, mixed precision, with grid barriers (cooperative launch, no
// clusters); its own unit so that the variants compile in parallel.
#include "minimize_launch.cuh"

namespace aqs {

cudaError_t run_mem_2_mixed_gb(int mem, const MinArgs* a, int n_clusters, int C, int npc,
                              size_t smem, cudaStream_t s, int* max_clusters) {
  return run_mem<2, true, 1, true>(mem, a, n_clusters, C, npc, smem, s, max_clusters);
}

}  // namespace aqs
