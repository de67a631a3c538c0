// sylv_dag_common.cuh -- grid sizing shared by the DAG launch units.
#pragma once

#include <cstdlib>

#include "sylv_dag.cuh"
#include "sylv_launch.h"

namespace sylv {

template <int TT, typename T, bool ROBUST>
cudaError_t launch_dag_impl(const Work& w, int max_tasks, cudaStream_t stream, int* per_sm_out = nullptr) {
  static int per_sm = -1;
  static int nsm = 0;
  const size_t smem = sizeof(DagSmem<TT, T>);
  if (per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(dag_kernel<TT, T, ROBUST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<TT, T, ROBUST>, kThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = nb > 0 ? nb : 1;
    // the workspace holds factor stores for kMaxCtasPerSm<T> CTAs per SM
    if (per_sm > max_ctas_per_sm<T>()) per_sm = max_ctas_per_sm<T>();
    // Experiment knob: SYLV_CTAS_PER_SM=1 keeps one CTA per SM (no FP64-pipe sharing).
    if (const char* env = std::getenv("SYLV_CTAS_PER_SM")) {
      const int v = std::atoi(env);
      if (v >= 1 && v < per_sm) per_sm = v;
    }
  }
  if (per_sm_out) *per_sm_out = per_sm;
  if (max_tasks <= 0) return cudaSuccess;
  int grid = nsm * per_sm;
  if (grid > max_tasks) grid = max_tasks;
  profile_begin(stream);
  dag_kernel<TT, T, ROBUST><<<grid, kThreads, smem, stream>>>(w);
  const cudaError_t e = cudaGetLastError();
  profile_end(stream);
  return e;
}

}  // namespace sylv
