// sylv_dag_f64.cu -- FP64 instantiations of the tile-DAG kernel (robust and
// non-robust, tile capacities 32 and 64).
#include "sylv_dag_common.cuh"
#include "sylv_launch.h"

namespace sylv {

// Optional: update GEMMs yield the SM to a diagonal solve running on it (FP64 pipe
// contention on the critical path).  Off by default (measured no gain at
// m = n = 4000/8000 and a loss on the 4096-equation batch); SYLV_DIAG_PRIORITY=1
// enables it.
static int diag_priority() {
  static int v = -1;
  if (v < 0) {
    const char* env = std::getenv("SYLV_DIAG_PRIORITY");
    v = env ? (std::atoi(env) != 0) : 0;
  }
  return v;
}

cudaError_t launch_dag_f64(int tt, bool robust, const Work& w0, int max_tasks, cudaStream_t stream, int sm_limit) {
  Work w = w0;
  w.prio = diag_priority();
  w.sm_limit = sm_limit;
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
