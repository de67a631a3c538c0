// sylv_refine_batch.cuh -- FP32 + refinement for a batch of independent equations
// in one launch sequence: the same loop as the single-equation refinement
// (binary32 robust correction solves of A D + D B = R, X += D in binary64, the
// binary64-accurate residual R = C - A X - X B in double-float arithmetic on the
// binary32 pipes, then the recurrence R -= A D + D B), with every step batched
// over the equations.  Each equation keeps its own convergence state: once it has
// converged its residuals, conversions and accumulations are skipped, and the
// tile kernel passes over its tasks (Work::eqskip).  The launch sequence itself is
// fixed, so an execute can be captured in a CUDA graph.
#pragma once

#include "sylv_gemm.cuh"

namespace sylv {

// One equation of a batched refinement (device descriptor).  A, B are the binary64
// operands as the tile kernel sees them (anti-transposed / negated copies where
// op = T or isgn = -1); C is the caller's right-hand side (flipped in place for the
// transposed forms), overwritten by the solution.  Leading dimensions of the work
// arrays: m (Ah, Al, Rf, R, X, D) and n (Bh, Bl).
struct RefEq {
  int64_t m, n;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  float* Ah;
  float* Al;
  float* Bh;
  float* Bl;
  float* Rf;
  double* R;
  double* X;
  double* D;
  unsigned long long* slots;  // [0] max|A|, [1] max|B|, then (max|R|, max|D|, max|X|) per correction
  RefineState* rs;
  int32_t oz;                 // the first residual runs on the tensor cores (k_oz_gemm_batched)
  int32_t pad;
};

__device__ __forceinline__ unsigned long long* ref_slot(const RefEq& E, int it, int k) { return E.slots + 2 + 3 * it + k; }
__device__ __forceinline__ bool ref_done(const RefEq& E) { return ld_volatile(&E.rs->conv) != 0; }
// Scale exponent of the operand pair: from the larger of max|A|, max|B|.
__device__ __forceinline__ int ref_sa(const RefEq& E) {
  return norm_exp(E.slots[0] > E.slots[1] ? E.slots : E.slots + 1);
}

// Visits every (r, c) of a rows x cols column-major array from the CTAs along grid
// dimension x: a warp per column (coalesced along the rows), the warps of the grid
// strided over the columns; no index division.  Each lane loads four elements
// (load(r, c), a value) before it stores any (store(r, c, value)): the compiler may
// not move a load above a store that might alias it, so element by element every
// access would wait for the one before.
template <typename LD, typename ST>
__device__ __forceinline__ void for_each_rc(int64_t rows, int64_t cols, LD&& load, ST&& store) {
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < cols; c += nw)
    for (int64_t r0 = lane; r0 < rows; r0 += 128) {
      decltype(load(r0, c)) v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + 32 * u < rows) v[u] = load(r0 + 32 * u, c);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + 32 * u < rows) store(r0 + 32 * u, c, v[u]);
    }
}

// max |A| and max |B| over the quasi-triangular parts (equation blockIdx.y).
__global__ void k_bref_maxabs(const RefEq* __restrict__ eq) {
  const RefEq E = eq[blockIdx.y];
  unsigned long long ma = 0, mb = 0;  // maxima as bit patterns of |value| (abs_key)
  for_each_rc(
      E.m, E.m, [&](int64_t r, int64_t c) { return r <= c + 1 ? E.A[r + c * E.lda] : 0.0; },
      [&](int64_t, int64_t, double v) { ma = max(ma, abs_key(v)); });
  for_each_rc(
      E.n, E.n, [&](int64_t r, int64_t c) { return r <= c + 1 ? E.B[r + c * E.ldb] : 0.0; },
      [&](int64_t, int64_t, double v) { mb = max(mb, abs_key(v)); });
  ma = warp_max_key(ma);
  mb = warp_max_key(mb);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(E.slots, ma);
    atomicMax(E.slots + 1, mb);
  }
}

// (Ah, Al) and (Bh, Bl): binary32 pairs of A 2^-s and B 2^-s, quasi-triangular parts.
__global__ void k_bref_split(const RefEq* __restrict__ eq) {
  const RefEq E = eq[blockIdx.y];
  const int s = ref_sa(E);
  for_each_rc(
      E.m, E.m, [&](int64_t r, int64_t c) { return r <= c + 1 ? E.A[r + c * E.lda] : 0.0; },
      [&](int64_t r, int64_t c, double v) {
        const DF d = split_df_mul2(v, -s);
        E.Ah[r + c * E.m] = d.hi;
        E.Al[r + c * E.m] = d.lo;
      });
  for_each_rc(
      E.n, E.n, [&](int64_t r, int64_t c) { return r <= c + 1 ? E.B[r + c * E.ldb] : 0.0; },
      [&](int64_t r, int64_t c, double v) {
        const DF d = split_df_mul2(v, -s);
        E.Bh[r + c * E.n] = d.hi;
        E.Bl[r + c * E.n] = d.lo;
      });
}

// First right-hand side: R = C (X = 0), and max |C|.
__global__ void k_bref_copy_max(const RefEq* __restrict__ eq) {
  const RefEq E = eq[blockIdx.y];
  unsigned long long mx = 0;
  for_each_rc(
      E.m, E.n, [&](int64_t r, int64_t c) { return E.C[r + c * E.ldc]; },
      [&](int64_t r, int64_t c, double v) {
        E.R[r + c * E.m] = v;
        mx = max(mx, abs_key(v));
      });
  mx = warp_max_key(mx);
  if ((threadIdx.x & 31) == 0) atomicMax(ref_slot(E, 0, 0), mx);
}

// Residual before correction `it` (>= 1), one 64 x 64 tile per CTA (equation
// blockIdx.z): it == 1 the binary64-accurate R = C - A X - X B, later the
// recurrence R -= A D + D B with the last correction D.
__global__ void __launch_bounds__(256) k_bref_residual(const RefEq* __restrict__ eq, int it) {
  const RefEq E = eq[blockIdx.z];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * GT, j0 = static_cast<int64_t>(blockIdx.y) * GT;
  if (i0 >= E.m || j0 >= E.n || ref_done(E) || (it == 1 && E.oz)) return;
  if (it == 1)
    residual_df_tile(E.Ah, E.Al, E.m, E.Bh, E.Bl, E.n, E.C, E.ldc, E.X, E.m, E.R, E.m, E.m, E.n, E.slots,
                     E.slots + 1, ref_slot(E, it - 1, 2), ref_slot(E, it, 0), i0, j0);
  else
    residual_update_tile(E.Ah, E.m, E.Bh, E.n, E.D, E.m, E.R, E.m, E.m, E.n, E.slots, E.slots + 1,
                         ref_slot(E, it - 1, 1), ref_slot(E, it, 0), i0, j0);
}

// Right-hand side of correction `it` in binary32: Rf = R 2^-s, s from max |R|.
__global__ void k_bref_to_float(const RefEq* __restrict__ eq, int it) {
  const RefEq E = eq[blockIdx.y];
  if (ref_done(E)) return;
  const int s = norm_exp(ref_slot(E, it, 0));
  for_each_rc(
      E.m, E.n, [&](int64_t r, int64_t c) { return E.R[r + c * E.m]; },
      [&](int64_t r, int64_t c, double v) { E.Rf[r + c * E.m] = f32_mul2(v, -s); });
}

// X += D per solved tile (the correction solve left tile (k,l) of D' = 2^(sa-sr) D as
// 2^e_kl-scaled floats in Rf), D kept for the next residual; max |D| and max |X| per
// equation.  Tasks of converged equations are passed over.
__global__ void k_bref_accumulate(Work wf, const RefEq* __restrict__ eq, int it) {
  const int ntasks = wf.ctrl->ntasks;
  for (int idx = blockIdx.x; idx < ntasks; idx += gridDim.x) {
    const Task tk = wf.tasks[idx];
    const RefEq E = eq[tk.inst];
    if (ref_done(E)) continue;  // uniform over the CTA: one task per iteration
    const Inst I = wf.inst[tk.inst];
    const int sr = norm_exp(ref_slot(E, it, 0));
    const int sa = ref_sa(E);
    const int e = wf.texp[I.tile + tk.tile];
    const int k = tk.tile / I.qmax, l = tk.tile % I.qmax;
    const int32_t* rb = wf.ibuf + I.rb;
    const int32_t* cb = wf.ibuf + I.cb;
    const int r0 = rb[k], mt = rb[k + 1] - r0, c0 = cb[l], nt = cb[l + 1] - c0;
    unsigned long long md = 0, mxv = 0;  // abs_key maxima
    // loads of four elements before their stores (see for_each_rc)
    for (int i0 = threadIdx.x; i0 < mt * nt; i0 += 4 * blockDim.x) {
      float rf[4];
      double xo[4];
      int64_t xi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        xi[u] = i < mt * nt ? (r0 + i % mt) + static_cast<int64_t>(c0 + i / mt) * E.m : -1;
        rf[u] = xi[u] >= 0 ? E.Rf[xi[u]] : 0.0f;
        xo[u] = xi[u] >= 0 ? E.X[xi[u]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (xi[u] >= 0) {
          const double dv = f64_mul2(rf[u], sr - sa - e);
          const double xv = xo[u] + dv;
          E.X[xi[u]] = xv;
          E.D[xi[u]] = dv;
          md = max(md, abs_key(dv));
          mxv = max(mxv, abs_key(xv));
        }
    }
    md = warp_max_key(md);
    mxv = warp_max_key(mxv);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(ref_slot(E, it, 1), md);
      atomicMax(ref_slot(E, it, 2), mxv);
    }
  }
}

// Convergence check after correction `it`, one thread per equation.  counters[0]
// counts arrivals and counters[1] converged equations (both zeroed before the
// launch); the last thread to arrive sets counters[2] once every equation has
// converged, which lets later tile-kernel launches return at once.
__global__ void k_bref_check(const RefEq* __restrict__ eq, int count, int it, double tol, Work wf, int* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const RefEq E = eq[i];
  const int err = wf.ctrl->err ? wf.ctrl->err : wf.st[i].err;
  refine_check_one(E.rs, ref_slot(E, it, 1), ref_slot(E, it, 2), it > 0 ? ref_slot(E, it - 1, 1) : nullptr, tol, err);
  if (E.rs->conv) atomicAdd(&counters[1], 1);
  __threadfence();
  if (atomicAdd(&counters[0], 1) == count - 1) {
    __threadfence();
    if (atomicAdd(&counters[1], 0) == count) atomicExch(&counters[2], 1);
  }
}

// C = X and the result record of each equation (equation blockIdx.y); an equation
// whose refinement overflowed keeps its right-hand side in C.
__global__ void k_bref_finish(const RefEq* __restrict__ eq, sylv_result* res) {
  const RefEq E = eq[blockIdx.y];
  if (E.rs->err != SYLV_OVERFLOWED)
    for_each_rc(
      E.m, E.n, [&](int64_t r, int64_t c) { return E.X[r + c * E.m]; },
      [&](int64_t r, int64_t c, double v) { E.C[r + c * E.ldc] = v; });
  if (blockIdx.x == 0 && threadIdx.x == 0) refine_result_one(E.rs, res + blockIdx.y);
}

// Row (dim 0) or column (dim 1) reversal of each equation's C in place.
__global__ void k_bref_flip(const RefEq* __restrict__ eq, int dim) {
  const RefEq E = eq[blockIdx.y];
  const int64_t m = E.m, n = E.n;
  const int64_t half = dim == 0 ? (m / 2) * n : m * (n / 2);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < half;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t i, j, i2, j2;
    if (dim == 0) {
      i = t % (m / 2);
      j = t / (m / 2);
      i2 = m - 1 - i;
      j2 = j;
    } else {
      i = t % m;
      j = t / m;
      i2 = i;
      j2 = n - 1 - j;
    }
    const double a = E.C[i + j * E.ldc], b = E.C[i2 + j2 * E.ldc];
    E.C[i + j * E.ldc] = b;
    E.C[i2 + j2 * E.ldc] = a;
  }
}

}  // namespace sylv
