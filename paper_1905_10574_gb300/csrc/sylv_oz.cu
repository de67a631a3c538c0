// sylv_oz.cu -- host side of the tensor-core residual (see sylv_oz.cuh): workspace
// sizes, the splitting launches and the GEMM launch.
#include <algorithm>

#include "sylv_launch.h"
#include "sylv_oz.cuh"

namespace sylv {

namespace {
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Packed views of the four operands: A (left of A X), X by columns (right of A X),
// X by rows (left of X B), B by columns (right of X B).
void shapes(int64_t m, int64_t n, oz::Packed (&P)[4]) {
  P[0] = {nullptr, nullptr, cdiv(m, oz::BM), cdiv(m, oz::BK), oz::BM};
  P[1] = {nullptr, nullptr, cdiv(n, oz::BN), cdiv(m, oz::BK), oz::BN};
  P[2] = {nullptr, nullptr, cdiv(m, oz::BM), cdiv(n, oz::BK), oz::BM};
  P[3] = {nullptr, nullptr, cdiv(n, oz::BN), cdiv(n, oz::BK), oz::BN};
}

int grid_elems(int64_t count) { return static_cast<int>(std::min<int64_t>(cdiv(count, 256), 152 * 16)); }
}  // namespace

size_t oz_workspace_bytes(int64_t m, int64_t n) {
  oz::Packed P[4];
  shapes(m, n, P);
  size_t tot = 0;
  for (auto& p : P) tot += up256(sizeof(__nv_bfloat16) * oz::kSlices * p.slice_elems()) + up256(sizeof(int) * p.RB * p.R);
  return tot;
}

void oz_carve(char* base, int64_t m, int64_t n, OzBuffers* b) {
  oz::Packed P[4];
  shapes(m, n, P);
  size_t off = 0;
  for (int i = 0; i < 4; ++i) {
    b->p[i] = base + off;
    off += up256(sizeof(__nv_bfloat16) * oz::kSlices * P[i].slice_elems());
    b->e[i] = reinterpret_cast<int*>(base + off);
    off += up256(sizeof(int) * P[i].RB * P[i].R);
  }
  b->m = m;
  b->n = n;
}

namespace {
oz::Packed packed(const OzBuffers& b, int i) {
  oz::Packed P[4];
  shapes(b.m, b.n, P);
  P[i].p = static_cast<__nv_bfloat16*>(b.p[i]);
  P[i].e = b.e[i];
  return P[i];
}
cudaError_t split(const oz::View& v, const oz::Packed& P, const int* skip, cudaStream_t s) {
  oz::k_oz_rowexp<<<grid_elems(P.RB * P.R * 32), 256, 0, s>>>(v, P.e, P.RB * P.R, skip);
  oz::k_oz_split<<<static_cast<int>(std::min<int64_t>(P.RB * P.KB, 152 * 8)), 256, 0, s>>>(v, P, skip);
  return cudaGetLastError();
}
}  // namespace

cudaError_t oz_split_ab(const OzBuffers& b, const double* A, int64_t lda, const double* B, int64_t ldb,
                        const int* skip, cudaStream_t s) {
  // A as rows (mask: r <= k + 1); B by columns: element (j, k) = B[k, j], kept for k <= j + 1.
  const oz::View va{A, 1, lda, b.m, b.m, 1};
  const oz::View vb{B, ldb, 1, b.n, b.n, 2};
  cudaError_t e = split(va, packed(b, 0), skip, s);
  if (e == cudaSuccess) e = split(vb, packed(b, 3), skip, s);
  return e;
}

cudaError_t oz_residual(const OzBuffers& b, const double* X, int64_t ldx, const double* C, int64_t ldc, double* R,
                        int64_t ldr, unsigned long long* rmax, int* err, long long timeout_ns, const int* skip,
                        cudaStream_t s, bool binary64) {
  const int64_t m = b.m, n = b.n;
  const oz::View vxc{X, ldx, 1, n, m, 0};  // X by columns: element (j, i) = X[i, j]
  const oz::View vxr{X, 1, ldx, m, n, 0};  // X by rows: element (i, j) = X[i, j]
  cudaError_t e = split(vxc, packed(b, 1), skip, s);
  if (e == cudaSuccess) e = split(vxr, packed(b, 2), skip, s);
  if (e != cudaSuccess) return e;
  oz::Gemm g;
  g.a[0] = packed(b, 0);
  g.b[0] = packed(b, 1);
  g.a[1] = packed(b, 2);
  g.b[1] = packed(b, 3);
  g.dense = 0;
  auto kern = binary64 ? oz::k_oz_gemm<oz::kMaxW> : oz::k_oz_gemm<oz::kMaxW32>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sizeof(oz::Smem)));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(cdiv(m, oz::BM)), static_cast<unsigned>(cdiv(n, oz::BN)));
  kern<<<grid, oz::kThreads, sizeof(oz::Smem), s>>>(g, C, ldc, R, ldr, m, n, rmax, err, timeout_ns, skip);
  return cudaGetLastError();
}

// ---- batched residuals (FP32 + refinement of many equations)
cudaError_t oz_batch_split(const OzBatchEq* eqs, int count, unsigned mask, int64_t max_rows, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  // rows: a warp each (8 per CTA); tiles: a CTA each, both strided over <= 64 CTAs per equation
  const unsigned gr = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cdiv(max_rows + oz::BM, 8), 64)));
  const unsigned gt = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>(cdiv(max_rows, oz::BN) * cdiv(max_rows, oz::BK), 64)));
  for (int which = 0; which < 4; ++which) {
    if (!(mask & (1u << which))) continue;
    oz::k_oz_rowexp_batched<<<dim3(gr, count), 256, 0, s>>>(eqs, which);
    oz::k_oz_split_batched<<<dim3(gt, count), 256, 0, s>>>(eqs, which);
  }
  return cudaGetLastError();
}

cudaError_t oz_batch_residual(const OzBatchEq* eqs, const OzTask* tasks, int ntasks, int* err, long long timeout_ns,
                              cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  auto kern = oz::k_oz_gemm_batched<oz::kMaxW>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sizeof(oz::Smem)));
  if (e != cudaSuccess) return e;
  kern<<<ntasks, oz::kThreads, sizeof(oz::Smem), s>>>(eqs, tasks, err, timeout_ns);
  return cudaGetLastError();
}

void oz_batch_tasks(int32_t eq, int64_t m, int64_t n, std::vector<OzTask>* out) {
  for (int64_t nb = 0; nb < cdiv(n, oz::BN); ++nb)
    for (int64_t mb = 0; mb < cdiv(m, oz::BM); ++mb)
      out->push_back(OzTask{eq, static_cast<int16_t>(mb), static_cast<int16_t>(nb)});
}

// ---- dense products (the Bartels-Stewart transformations)
namespace {
oz::Packed dense_left(int64_t rows, int64_t k) { return {nullptr, nullptr, cdiv(rows, oz::BM), cdiv(k, oz::BK), oz::BM}; }
oz::Packed dense_right(int64_t rows, int64_t k) { return {nullptr, nullptr, cdiv(rows, oz::BN), cdiv(k, oz::BK), oz::BN}; }
size_t packed_bytes(const oz::Packed& P) {
  return up256(sizeof(__nv_bfloat16) * oz::kSlices * P.slice_elems()) + up256(sizeof(int) * P.RB * P.R);
}
}  // namespace

size_t oz_dense_bytes(int64_t mo, int64_t no, int64_t kmax) {
  return packed_bytes(dense_left(mo, kmax)) + packed_bytes(dense_right(no, kmax));
}

cudaError_t oz_product(char* buf, const double* L, int64_t lrs, int64_t lks, const double* Q, int64_t qrs,
                       int64_t qks, int64_t mo, int64_t no, int64_t k, double* R, int64_t ldr, int* err,
                       long long timeout_ns, cudaStream_t s) {
  oz::Packed pl = dense_left(mo, k), pr = dense_right(no, k);
  pl.p = reinterpret_cast<__nv_bfloat16*>(buf);
  pl.e = reinterpret_cast<int*>(buf + up256(sizeof(__nv_bfloat16) * oz::kSlices * pl.slice_elems()));
  char* rb = buf + packed_bytes(pl);
  pr.p = reinterpret_cast<__nv_bfloat16*>(rb);
  pr.e = reinterpret_cast<int*>(rb + up256(sizeof(__nv_bfloat16) * oz::kSlices * pr.slice_elems()));
  const oz::View vl{L, lrs, lks, mo, k, 0};
  const oz::View vq{Q, qrs, qks, no, k, 0};
  cudaError_t e = split(vl, pl, nullptr, s);
  if (e == cudaSuccess) e = split(vq, pr, nullptr, s);
  if (e != cudaSuccess) return e;
  oz::Gemm g;
  g.a[0] = g.a[1] = pl;
  g.b[0] = g.b[1] = pr;
  g.dense = 1;
  auto kern = oz::k_oz_gemm<oz::kMaxW>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sizeof(oz::Smem)));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(cdiv(mo, oz::BM)), static_cast<unsigned>(cdiv(no, oz::BN)));
  kern<<<grid, oz::kThreads, sizeof(oz::Smem), s>>>(g, R, ldr, R, ldr, mo, no, nullptr, err, timeout_ns, nullptr);
  return cudaGetLastError();
}

}  // namespace sylv
