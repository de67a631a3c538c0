// sylv_dag_f64.cu -- FP64 instantiations of the tile-DAG kernel (robust and
// non-robust, tile capacities 32 and 64).
#include "sylv_dag_common.cuh"
#include "sylv_launch.h"

namespace sylv {

cudaError_t launch_dag_f64(int tt, bool robust, const Work& w, int max_tasks, cudaStream_t stream) {
  if (tt <= 32) return robust ? launch_dag_impl<32, double, true>(w, max_tasks, stream)
                              : launch_dag_impl<32, double, false>(w, max_tasks, stream);
  return robust ? launch_dag_impl<64, double, true>(w, max_tasks, stream)
                : launch_dag_impl<64, double, false>(w, max_tasks, stream);
}

int dag_ctas_per_sm_f64(int tt, bool robust) {
  int n = 0;
  Work w{};
  if (tt <= 32)
    robust ? launch_dag_impl<32, double, true>(w, 0, 0, &n) : launch_dag_impl<32, double, false>(w, 0, 0, &n);
  else
    robust ? launch_dag_impl<64, double, true>(w, 0, 0, &n) : launch_dag_impl<64, double, false>(w, 0, 0, &n);
  return n;
}

}  // namespace sylv
