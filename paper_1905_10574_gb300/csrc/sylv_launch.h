// sylv_launch.h -- host-side launchers of the tile-DAG kernel instantiations
// (one translation unit per element type so that they compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "sylv_internal.cuh"

namespace sylv {

// CTAs per SM the tile kernel may use (and the workspace reserves factor stores for):
// 2 for the FP64 kernel (FP64-pipe bound), 4 for the FP32 correction solves
// (latency bound).
template <typename T>
constexpr int max_ctas_per_sm() {
  return sizeof(T) == 4 ? 4 : 2;
}

// Launch the persistent DAG kernel for tile capacity tt (32 or 64) on `stream`.
// max_tasks bounds the grid (no more CTAs than tiles).  Returns the launch error.
cudaError_t launch_dag_f64(int tt, bool robust, const Work& w, int max_tasks, cudaStream_t stream);
cudaError_t launch_dag_f32(int tt, const Work& w, int max_tasks, cudaStream_t stream);

// Event bracketing of DAG launches for sylv_profile (no-ops unless enabled).
void profile_begin(cudaStream_t stream);
void profile_end(cudaStream_t stream);

// Resident CTAs per SM of an instantiation (for reporting and grid sizing).
int dag_ctas_per_sm_f64(int tt, bool robust);

}  // namespace sylv
