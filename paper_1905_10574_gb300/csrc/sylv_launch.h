// sylv_launch.h -- host-side launchers of the tile-DAG kernel instantiations
// (one translation unit per element type so that they compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "sylv_internal.cuh"

namespace sylv {

// CTAs per SM the tile kernel may use (and the workspace reserves factor stores for):
// both instantiations hold 2 per SM (registers and shared memory).
template <typename T>
constexpr int max_ctas_per_sm() {
  return 2;
}

// Launch the persistent DAG kernel for tile capacity tt (32 or 64) on `stream`.
// max_tasks bounds the grid (no more CTAs than tiles).  Returns the launch error.
// sm_limit > 0 runs the tile kernel on the SMs with id < sm_limit only (SM scaling).
cudaError_t launch_dag_f64(int tt, bool robust, const Work& w, int max_tasks, cudaStream_t stream, int sm_limit = 0);
cudaError_t launch_dag_f32(int tt, const Work& w, int max_tasks, cudaStream_t stream, int sm_limit = 0);

// Event bracketing of DAG launches for sylv_profile (no-ops unless enabled).
void profile_begin(cudaStream_t stream);
void profile_end(cudaStream_t stream);

// Resident CTAs per SM of an instantiation (for reporting and grid sizing).
int dag_ctas_per_sm_f64(int tt, bool robust);

// Tensor-core residual R = C - (A X + X B) of the refinement (sylv_oz.cuh): operand
// slices in four packed arrays (A; X by columns; X by rows; B by columns) with their
// per-row exponents.
struct OzBuffers {
  void* p[4];
  int* e[4];
  int64_t m, n;
};
size_t oz_workspace_bytes(int64_t m, int64_t n);
void oz_carve(char* base, int64_t m, int64_t n, OzBuffers* b);
// Slices of A and B (once per solve).
cudaError_t oz_split_ab(const OzBuffers& b, const double* A, int64_t lda, const double* B, int64_t ldb,
                        const int* skip, cudaStream_t s);
// Slices of X, then R = C - (A X + X B) and max |R| (into rmax); a timeout sets *err.
// binary64: all slice pairs of the binary64-accurate residual; otherwise the pairs of
// a binary32-accurate product.  R may equal C (in place).
cudaError_t oz_residual(const OzBuffers& b, const double* X, int64_t ldx, const double* C, int64_t ldc, double* R,
                        int64_t ldr, unsigned long long* rmax, int* err, long long timeout_ns, const int* skip,
                        cudaStream_t s, bool binary64);
// Batched form: one equation's operands, outputs and packed slices (oz_carve).
struct OzBatchEq {
  OzBuffers b;  // packed slices and exponents; b.m, b.n the equation's orders
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  const double* X;  // the current solution, m x n
  int64_t ldx;
  const double* C;
  int64_t ldc;
  double* R;        // R = C - (A X + X B)
  int64_t ldr;
  unsigned long long* rmax;  // max |R| of the equation (atomic maximum of the bit patterns)
  const int* skip;           // nonzero: the equation is passed over (converged)
  int32_t active;            // 0: the equation takes another residual (the kernels pass it over)
  int32_t pad;
};
// One 128 x 64 output tile of one equation.
struct OzTask {
  int32_t eq;
  int16_t mb, nb;
};
// Slices of the operands in `mask` (bit 0 A, 1 X by columns, 2 X by rows, 3 B) of
// every equation; max_rows / max_k bound every equation's orders.
cudaError_t oz_batch_split(const OzBatchEq* eqs, int count, unsigned mask, int64_t max_rows, cudaStream_t s);
// R = C - (A X + X B) and max |R| for every task's tile (binary64-accurate).
cudaError_t oz_batch_residual(const OzBatchEq* eqs, const OzTask* tasks, int ntasks, int* err, long long timeout_ns,
                              cudaStream_t s);
// The tasks of an equation of orders m x n (appended to `out`).
void oz_batch_tasks(int32_t eq, int64_t m, int64_t n, std::vector<OzTask>* out);

// Dense product on the same tensor-core kernel, binary64-accurate (error-free
// splitting): R -= L Q^T for L (mo x k, element (r, c) at L[r lrs + c lks]) and Q
// (no x k, element (j, c) at Q[j qrs + c qks]); R is mo x no with leading dimension
// ldr.  buf: oz_dense_bytes(mo, no, k') bytes for any k' >= k; a timeout sets *err.
size_t oz_dense_bytes(int64_t mo, int64_t no, int64_t kmax);
cudaError_t oz_product(char* buf, const double* L, int64_t lrs, int64_t lks, const double* Q, int64_t qrs,
                       int64_t qks, int64_t mo, int64_t no, int64_t k, double* R, int64_t ldr, int* err,
                       long long timeout_ns, cudaStream_t s);

}  // namespace sylv
