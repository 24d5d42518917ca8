// launch.cuh -- kernel launch bookkeeping shared by the library's sources.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aqs {
// Counts every kernel launch the library makes (reported by aqs_launch_count).
void count_launch();
}  // namespace aqs
