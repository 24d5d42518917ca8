// launch.cuh -- kernel launch bookkeeping shared by the library's sources.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aqs {
// Counts every kernel launch the library makes (reported by aqs_launch_count).
void count_launch();
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount;
// 152 on GB300), used to size grids and clusters.
int sm_count();
}  // namespace aqs
