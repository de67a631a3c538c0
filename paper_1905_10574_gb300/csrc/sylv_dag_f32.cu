// sylv_dag_f32.cu -- FP32 instantiations of the tile-DAG kernel, used for the
// correction solves of the FP32 + refinement mode (robust; binary32 small solves
// with FP64 bound arithmetic and an FP64 guarded fallback).
#include "sylv_dag_common.cuh"
#include "sylv_launch.h"

namespace sylv {

cudaError_t launch_dag_f32(int tt, const Work& w0, int max_tasks, cudaStream_t stream, int sm_limit) {
  Work w = w0;
  w.sm_limit = sm_limit;
  if (tt <= 32) return launch_dag_impl<32, float, true>(w, max_tasks, stream);
  return launch_dag_impl<64, float, true>(w, max_tasks, stream);
}

}  // namespace sylv
