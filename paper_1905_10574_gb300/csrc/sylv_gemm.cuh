// sylv_gemm.cuh -- dense FP64 kernels around the solver: the residual
// R = C - A X - X B of the refinement loop, the gradient products of the adjoint,
// and the elementwise helpers of the FP32 + refinement mode.
#pragma once

#include "sylv_internal.cuh"

namespace sylv {

// Register-tiled FP64 tile: 64 x 64 outputs per CTA, 256 threads, 4 x 4 each,
// k-chunks of 16 staged in shared memory (k-major rows, 16-byte aligned).
constexpr int GT = 64, GK = 16, GLD = GT + 2;

// R = C - A X - X B for upper quasi-triangular A (m x m), B (n x n): only A[r,c]
// with r <= c+1 and B[r,c] with r <= c+1 take part (the entries the solver reads).
// Also records max |R| (bit pattern of a non-negative double) in *rmax.
// If *skip != 0 the kernel does nothing (the refinement has converged).
__global__ void __launch_bounds__(256) k_residual(const double* __restrict__ A, int64_t lda,
                                                  const double* __restrict__ B, int64_t ldb,
                                                  const double* __restrict__ C, int64_t ldc,
                                                  const double* __restrict__ X, int64_t ldx,
                                                  double* __restrict__ R, int64_t ldr, int64_t m, int64_t n,
                                                  unsigned long long* rmax, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  __shared__ __align__(16) double Ls[GK * GLD];
  __shared__ __align__(16) double Rs[GK * GLD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * GT, j0 = static_cast<int64_t>(blockIdx.y) * GT;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      acc[i][j] = (r < m && c < n) ? C[r + c * ldc] : 0.0;
    }
  // A X: k runs over columns of A that rows i0.. can touch: k >= i0 - 1.
  const int64_t ka = i0 > 0 ? i0 - 1 : 0;
  for (int64_t k0 = ka; k0 < m; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      Ls[kk * GLD + r] = (gr < m && gk < m && gr <= gk + 1) ? A[gr + gk * lda] : 0.0;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      Rs[kk2 * GLD + c] = (gk2 < m && gc < n) ? X[gk2 + gc * ldx] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ls[kk * GLD + tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Rs[kk * GLD + ty * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  // X B: k runs over rows of B that columns j0.. can touch: k <= j0 + GT.
  const int64_t kb_end = (j0 + GT + 1 < n) ? j0 + GT + 1 : n;
  for (int64_t k0 = 0; k0 < kb_end; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      Ls[kk * GLD + r] = (gr < m && gk < n) ? X[gr + gk * ldx] : 0.0;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      Rs[kk2 * GLD + c] = (gk2 < n && gc < n && gk2 <= gc + 1) ? B[gk2 + gc * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ls[kk * GLD + tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Rs[kk * GLD + ty * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      if (r < m && c < n) {
        R[r + c * ldr] = acc[i][j];
        mx = fmax(mx, fabs(acc[i][j]));
      }
    }
  mx = warp_max(mx);
  if ((tid & 31) == 0 && rmax) atomic_max_nonneg(rmax, mx);
}

// Exponent that undoes the adjoint solve's own scale 2^log2scale (rs: its device
// result record, null: none), clamped where every finite double is sent to 0 or Inf.
__device__ __forceinline__ int unscale_exp(const sylv_result* rs, int64_t extra) {
  const int64_t e = extra - (rs ? rs->log2scale : 0);
  return static_cast<int>(e < -4000 ? -4000 : (e > 4000 ? 4000 : e));
}
// v * 2^e; a finite v that leaves the binary64 range marks the record SYLV_OVERFLOWED.
__device__ __forceinline__ double unscale(double v, int e, sylv_result* rs) {
  const double r = mul2(v, e);
  if (rs && isfinite(v) && !isfinite(r)) atomicMax(&rs->info, SYLV_OVERFLOWED);
  return r;
}

// D = -P Q^T-like products for the adjoint: D[i,j] = -sum_c P(i,c) Q(j,c) with
// P(i,c) = P[i*psi + c*psc], Q(j,c) = Q[j*qsj + c*qsc] (element strides, so the
// same kernel serves Gamma Y^T, Y Gamma^T, Y^T Gamma and Gamma^T Y), masked to
// the entries a quasi-triangular operand T (N x N, ldt) exposes: i <= j, or
// i == j + 1 with T[i, j] != 0.  Other entries of D are set to 0.  With a result
// record rs, D is multiplied by 2^-rs->log2scale (exact), undoing the scale of the
// adjoint solve that produced P or Q.
__global__ void __launch_bounds__(256) k_grad_product(const double* __restrict__ P, int64_t psi, int64_t psc,
                                                      const double* __restrict__ Q, int64_t qsj, int64_t qsc,
                                                      int64_t N, int64_t K, const double* __restrict__ T,
                                                      int64_t ldt, double* __restrict__ D, int64_t ldd,
                                                      double sign, sylv_result* rs) {
  const int eu = unscale_exp(rs, 0);
  __shared__ __align__(16) double Ls[GK * GLD];
  __shared__ __align__(16) double Rs[GK * GLD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * GT, j0 = static_cast<int64_t>(blockIdx.y) * GT;
  const bool active = i0 <= j0 + GT;  // tile touches the upper quasi-triangle
  double acc[4][4] = {};
  if (active) {
    for (int64_t k0 = 0; k0 < K; k0 += GK) {
      for (int idx = tid; idx < GK * GT; idx += 256) {
        const int r = idx % GT, kk = idx / GT;
        const int64_t gi = i0 + r, gk = k0 + kk;
        Ls[kk * GLD + r] = (gi < N && gk < K) ? P[gi * psi + gk * psc] : 0.0;
        const int64_t gj = j0 + r;
        Rs[kk * GLD + r] = (gj < N && gk < K) ? Q[gj * qsj + gk * qsc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ls[kk * GLD + tx * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Rs[kk * GLD + ty * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      if (r < N && c < N) {
        const bool keep = (r <= c) || (r == c + 1 && T[r + c * ldt] != 0.0);
        D[r + c * ldd] = keep ? unscale(sign * acc[i][j], eu, rs) : 0.0;
      }
    }
}

// ---------------------------------------------------------------- refinement helpers
// max |T[r,c]| over the quasi-triangular part (r <= c+1) of an N x N matrix.
__global__ void k_maxabs_quasi(const double* __restrict__ T, int64_t ldt, int64_t N, unsigned long long* out) {
  double mx = 0.0;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < N * N;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % N, c = t / N;
    if (r <= c + 1) mx = fmax(mx, fabs(T[r + c * ldt]));
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, mx);
}

// Exponent s with max|.| * 2^-s in [1, 2): s = floor(log2(max)), 0 for a zero max.
__device__ __forceinline__ int norm_exp(const unsigned long long* slot) {
  const double v = __longlong_as_double(static_cast<long long>(*slot));
  return (v > 0.0 && v <= 1.7976931348623157e308) ? floor_log2(v) : 0;
}

// dst (float) = src * 2^-s, s from the larger of slot_a/slot_b (null = 0);
// quasi != 0 keeps only r <= c+1 (other entries 0).
__global__ void k_to_float(const double* __restrict__ src, int64_t lds, float* __restrict__ dst, int64_t ldd,
                           int64_t rows, int64_t cols, const unsigned long long* slot_a,
                           const unsigned long long* slot_b, int quasi, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  int s = 0;
  if (slot_a) {
    const unsigned long long a = *slot_a, b = slot_b ? *slot_b : 0ull;
    s = norm_exp(a > b ? slot_a : slot_b);
  }
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < rows * cols;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % rows, c = t / rows;
    const double v = (!quasi || r <= c + 1) ? src[r + c * lds] : 0.0;
    dst[r + c * ldd] = static_cast<float>(mul2(v, -s));
  }
}

// R = C (first refinement right-hand side, X = 0) and max |C|.
__global__ void k_copy_max(const double* __restrict__ C, int64_t ldc, double* __restrict__ R, int64_t ldr,
                           int64_t m, int64_t n, unsigned long long* rmax) {
  double mx = 0.0;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    const double v = C[r + c * ldc];
    R[r + c * ldr] = v;
    mx = fmax(mx, fabs(v));
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rmax, mx);
}

// X += D where the FP32 correction solve left tile (k,l) of D' = 2^(sa-sr) D as
// 2^e_kl-scaled floats in Rf: D = Rf * 2^(sr - sa - e_kl).  Records max|D|, max|X|.
__global__ void k_accumulate(Work wf, double* __restrict__ X, int64_t ldx, double* __restrict__ Dout,
                             const unsigned long long* slot_r, const unsigned long long* slot_a,
                             const unsigned long long* slot_b, unsigned long long* dmax, unsigned long long* xmax,
                             const int* skip) {
  if (skip && ld_volatile(skip)) return;
  const int sr = norm_exp(slot_r);
  const unsigned long long a = *slot_a, b = *slot_b;
  const int sa = norm_exp(a > b ? slot_a : slot_b);
  const int ntasks = wf.ctrl->ntasks;
  double md = 0.0, mxv = 0.0;
  for (int idx = blockIdx.x; idx < ntasks; idx += gridDim.x) {
    const Task tk = wf.tasks[idx];
    const Inst I = wf.inst[tk.inst];
    const int e = wf.texp[I.tile + tk.tile];
    const int k = tk.tile / I.qmax, l = tk.tile % I.qmax;
    const int32_t* rb = wf.ibuf + I.rb;
    const int32_t* cb = wf.ibuf + I.cb;
    const int r0 = rb[k], mt = rb[k + 1] - r0, c0 = cb[l], nt = cb[l + 1] - c0;
    const float* Rf = static_cast<const float*>(I.C);
    for (int i = threadIdx.x; i < mt * nt; i += blockDim.x) {
      const int64_t r = r0 + i % mt, c = c0 + i / mt;
      const double dv = mul2(static_cast<double>(Rf[r + c * I.ldc]), sr - sa - e);
      const double xv = X[r + c * ldx] + dv;
      X[r + c * ldx] = xv;
      if (Dout) Dout[r + c * ldx] = dv;
      md = fmax(md, fabs(dv));
      mxv = fmax(mxv, fabs(xv));
    }
  }
  md = warp_max(md);
  mxv = warp_max(mxv);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(dmax, md);
    atomic_max_nonneg(xmax, mxv);
  }
}

// After correction `it`: converged when max|D| <= tol * max|X| (or the FP32
// solve failed).  Updates the iteration count and the last ratio.
struct RefineState {
  int conv;
  int iters;
  int err;
  int pad;
  double last;
};
// After correction k: converged when max|D_k| <= tol max|X|, or when the
// corrections contract (ratio rho = max|D_k| / max|D_{k-1}| < 1/2) and the next one
// would be below the tolerance: rho max|D_k| <= tol max|X|.  dprev: previous max|D|
// slot (null for the first correction, which is the whole first solution).
// The check of one equation; err: the first error of its correction solve (0: none).
__device__ __forceinline__ void refine_check_one(RefineState* rs, const unsigned long long* dmax,
                                                 const unsigned long long* xmax, const unsigned long long* dprev,
                                                 double tol, int e) {
  if (rs->conv) return;
  const double d = __longlong_as_double(static_cast<long long>(*dmax));
  const double x = __longlong_as_double(static_cast<long long>(*xmax));
  rs->iters += 1;
  // The refined solution is returned at alpha = 1: a correction or a solution beyond
  // the binary64 range (infinite or NaN maximum) ends the loop with SYLV_OVERFLOWED,
  // and the equation's C is left as it was (the robust FP64 solve scales instead).
  if (!(d <= 1.7976931348623157e308) || !(x <= 1.7976931348623157e308)) {
    rs->err = SYLV_OVERFLOWED;
    rs->conv = 1;
    rs->last = 0.0;
    return;
  }
  rs->last = (x > 0.0) ? d / x : (d > 0.0 ? 1.0 : 0.0);
  bool conv = d <= tol * x;
  if (!conv && dprev) {
    const double dp = __longlong_as_double(static_cast<long long>(*dprev));
    const double rho = dp > 0.0 ? d / dp : 1.0;
    if (rho < 0.5 && rho * d <= tol * x) {
      conv = true;
      rs->last = rho * d / x;  // the predicted size of the next correction
    }
  }
  if (e) {
    rs->err = e;
    rs->conv = 1;
  } else {
    rs->conv = conv ? 1 : 0;
  }
}

__global__ void k_refine_check(RefineState* rs, const unsigned long long* dmax, const unsigned long long* xmax,
                               const unsigned long long* dprev, double tol, const Work wf) {
  refine_check_one(rs, dmax, xmax, dprev, tol, wf.ctrl->err ? wf.ctrl->err : wf.st[0].err);
}

__device__ __forceinline__ void refine_result_one(const RefineState* rs, sylv_result* res) {
  sylv_result r;
  r.log2scale = 0;
  r.scale = 1.0;
  r.iters = rs->iters;
  r.last_update = rs->last;
  r.scale_events = 0;
  r.min_tile_exp = 0;
  r.info = rs->err ? rs->err : (rs->conv ? SYLV_OK : SYLV_NOT_CONVERGED);
  *res = r;
}

__global__ void k_refine_result(const RefineState* rs, sylv_result* res, int maxit) { refine_result_one(rs, res); }

// C (m x n, ldc) <- X, unless the refinement overflowed (C keeps the right-hand side).
__global__ void k_refine_copy_out(const double* __restrict__ X, int64_t ldx, double* __restrict__ C, int64_t ldc,
                                  int64_t m, int64_t n, const RefineState* rs) {
  if (rs->err == SYLV_OVERFLOWED) return;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    C[r + c * ldc] = X[r + c * ldx];
  }
}

// Y (m x n, ldy) <- X.
__global__ void k_copy(const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy, int64_t m,
                       int64_t n) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    Y[r + c * ldy] = X[r + c * ldx];
  }
}

// M *= 2^e (in place).
__global__ void k_scale_pow2(double* M, int64_t ld, int64_t m, int64_t n, int e) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    M[r + c * ld] = mul2(M[r + c * ld], e);
  }
}

// M *= 2^(e - rs->log2scale) (in place, exact unless the range is left; see unscale).
__global__ void k_unscale_pow2(double* M, int64_t ld, int64_t m, int64_t n, int64_t e, sylv_result* rs) {
  const int eu = unscale_exp(rs, e);
  if (eu == 0) return;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    M[r + c * ld] = unscale(M[r + c * ld], eu, rs);
  }
}

}  // namespace sylv

namespace sylv {

// ---------------------------------------------------------------- double-float residual
// Binary64-accurate products on the binary32 pipes (GB300 runs FP32 FMA at 64x
// the FP64 rate).  A value v is carried as a pair of floats (hi, lo), hi = fl32(v),
// lo = fl32(v - hi), ~48 significant bits.  For a term a*x:
//   p = ah*xh exactly as p + q with q = fma(ah, xh, -p)      (error-free product)
//   c = ah*xl + al*xh                                         (cross terms, fp32)
// and p enters the running sum s by Knuth's two-sum (s + p = s' + e exactly), while
// q, c and e go to a compensation accumulator.  Relative error of a sum of K terms
// ~ K * 2^-48 of sum |a||x| (each dropped al*xl is 2^-48 |a||x|).
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF split_df(double v) {
  const float h = static_cast<float>(v);
  return DF{h, static_cast<float>(v - static_cast<double>(h))};
}
// The same conversions from the bit patterns, for elementwise kernels: on this GPU
// every binary64 instruction (a multiply by 2^e, a conversion, a maximum) runs at
// 1/64 of the binary32 rate, so one per element already costs as much time as the
// element's memory traffic.  Results are those of the arithmetic forms; values
// outside the binary32 normal range take the arithmetic path.
//   f32_mul2(v, e)      = (float)(v 2^e), rounded to nearest even
//   split_df_mul2(v, e) = split_df(v 2^e)
//   f64_mul2(f, e)      = (double)f 2^e
//   abs_key(v)          = a key that orders |v| like the values (NaN above infinity)
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}
__device__ __forceinline__ float f32_mul2(double v, int e) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  if ((b << 1) == 0) return __uint_as_float(static_cast<unsigned>(b >> 32));  // signed zero
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  const int Ef = E - 896 + e;  // binary32 biased exponent before rounding
  if (E == 0 || E == 0x7ff || Ef <= 0 || Ef >= 254) return static_cast<float>(mul2(v, e));
  const unsigned keep = static_cast<unsigned>((b >> 29) & 0x7fffff);
  const unsigned rem = static_cast<unsigned>(b & 0x1fffffff);
  unsigned r = (static_cast<unsigned>(Ef) << 23) | keep;
  if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) r += 1;  // a carry moves into the exponent
  return __uint_as_float(r | (static_cast<unsigned>(b >> 32) & 0x80000000u));
}
__device__ __forceinline__ DF split_df_mul2(double v, int e) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  if ((b << 1) == 0) return DF{__uint_as_float(static_cast<unsigned>(b >> 32)), 0.0f};
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  const int Ef = E - 896 + e;
  if (E == 0 || E == 0x7ff || Ef <= 0 || Ef >= 254) return split_df(mul2(v, e));
  const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
  const unsigned keep = static_cast<unsigned>((b >> 29) & 0x7fffff);
  int rem = static_cast<int>(b & 0x1fffffff);
  unsigned r = (static_cast<unsigned>(Ef) << 23) | keep;
  if (rem > 0x10000000 || (rem == 0x10000000 && (keep & 1u))) {
    r += 1;
    rem -= 0x20000000;  // the remainder below the rounded-up high part
  }
  // v 2^e - hi = +-rem 2^(Ef - 179) (units of the binary64 significand's last bit, 29
  // below binary32's 2^(Ef - 150)): an integer below 2^29 converted with one rounding
  const float lo = mul2(static_cast<float>(sign ? -rem : rem), Ef - 179);
  return DF{__uint_as_float(r | sign), lo};
}
__device__ __forceinline__ double f64_mul2(float f, int e) {
  const unsigned b = __float_as_uint(f);
  const int Ef = static_cast<int>((b >> 23) & 0xff);
  const int Ed = Ef + 896 + e;
  if (Ef == 0 || Ef == 255 || Ed <= 0 || Ed >= 2047) return mul2(static_cast<double>(f), e);
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                                                     (static_cast<unsigned long long>(Ed) << 52) |
                                                     (static_cast<unsigned long long>(b & 0x7fffffu) << 29)));
}
__device__ __forceinline__ void df_acc(float& s, float& comp, float ah, float al, float xh, float xl) {
  const float p = ah * xh;
  const float q = fmaf(ah, xh, -p);
  float c = fmaf(ah, xl, q);
  c = fmaf(al, xh, c);
  const float t = s + p;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (p - bp);
  s = t;
  comp += e + c;
}

// R = C - A X - X B in binary64-accurate double-float arithmetic.  A (m x m) and B
// (n x n) are given as float pairs scaled by 2^-sa (sa from the max |entry| of A
// and B: AS = A 2^-sa, BS = B 2^-sa), restricted to their quasi-triangular parts;
// X (binary64) is scaled by 2^-sx (sx from max |X|) and split on the fly.  The
// kernel computes RS = C 2^-(sa+sx) - (AS XS + XS BS) = R 2^-(sa+sx) and stores
// R = RS 2^(sa+sx) in binary64, plus max |R| in *rmax.  64 x 64 output tile per CTA,
// 256 threads, 4 x 4 outputs each; k-chunks of 16 in shared memory.
// One 64 x 64 output tile (rows i0.., columns j0..) of k_residual_df.
__device__ __forceinline__ void residual_df_tile(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                 int64_t lda, const float* __restrict__ Bh,
                                                 const float* __restrict__ Bl, int64_t ldb,
                                                 const double* __restrict__ C, int64_t ldc,
                                                 const double* __restrict__ X, int64_t ldx,
                                                 double* __restrict__ R, int64_t ldr, int64_t m, int64_t n,
                                                 const unsigned long long* slot_a, const unsigned long long* slot_b,
                                                 const unsigned long long* slot_x, unsigned long long* rmax,
                                                 int64_t i0, int64_t j0) {
  constexpr int LD = GT + 4;  // float rows, 16-byte aligned
  __shared__ __align__(16) float Lh[GK * LD], Ll[GK * LD], Rh[GK * LD], Rl[GK * LD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const unsigned long long ua = *slot_a, ub = *slot_b;
  const int sa = norm_exp(ua > ub ? slot_a : slot_b);
  const int sx = norm_exp(slot_x);
  float s[4][4], comp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s[i][j] = 0.f;
      comp[i][j] = 0.f;
    }
  // A X part: k >= i0 - 1 (A quasi-upper-triangular).
  const int64_t ka = i0 > 0 ? i0 - 1 : 0;
  for (int64_t k0 = ka; k0 < m; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      const bool ok = gr < m && gk < m && gr <= gk + 1;
      Lh[kk * LD + r] = ok ? Ah[gr + gk * lda] : 0.f;
      Ll[kk * LD + r] = ok ? Al[gr + gk * lda] : 0.f;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      const DF x = (gk2 < m && gc < n) ? split_df(mul2(X[gk2 + gc * ldx], -sx)) : DF{0.f, 0.f};
      Rh[kk2 * LD + c] = x.hi;
      Rl[kk2 * LD + c] = x.lo;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      float ah[4], al[4], xh[4], xl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Lh[kk * LD + tx * 4 + i];
        al[i] = Ll[kk * LD + tx * 4 + i];
        xh[i] = Rh[kk * LD + ty * 4 + i];
        xl[i] = Rl[kk * LD + ty * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_acc(s[i][j], comp[i][j], ah[i], al[i], xh[j], xl[j]);
    }
    __syncthreads();
  }
  // X B part: k <= j0 + GT (B quasi-upper-triangular).
  const int64_t kb_end = (j0 + GT + 1 < n) ? j0 + GT + 1 : n;
  for (int64_t k0 = 0; k0 < kb_end; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      const DF x = (gr < m && gk < n) ? split_df(mul2(X[gr + gk * ldx], -sx)) : DF{0.f, 0.f};
      Lh[kk * LD + r] = x.hi;
      Ll[kk * LD + r] = x.lo;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      const bool ok = gk2 < n && gc < n && gk2 <= gc + 1;
      Rh[kk2 * LD + c] = ok ? Bh[gk2 + gc * ldb] : 0.f;
      Rl[kk2 * LD + c] = ok ? Bl[gk2 + gc * ldb] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      float xh[4], xl[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xh[i] = Lh[kk * LD + tx * 4 + i];
        xl[i] = Ll[kk * LD + tx * 4 + i];
        bh[i] = Rh[kk * LD + ty * 4 + i];
        bl[i] = Rl[kk * LD + ty * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_acc(s[i][j], comp[i][j], xh[i], xl[i], bh[j], bl[j]);
    }
    __syncthreads();
  }
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      if (r < m && c < n) {
        const double prod = static_cast<double>(s[i][j]) + static_cast<double>(comp[i][j]);
        const double v = C[r + c * ldc] - mul2(prod, sa + sx);
        R[r + c * ldr] = v;
        mx = fmax(mx, fabs(v));
      }
    }
  mx = warp_max(mx);
  if ((tid & 31) == 0 && rmax) atomic_max_nonneg(rmax, mx);
}

__global__ void __launch_bounds__(256) k_residual_df(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                     int64_t lda, const float* __restrict__ Bh,
                                                     const float* __restrict__ Bl, int64_t ldb,
                                                     const double* __restrict__ C, int64_t ldc,
                                                     const double* __restrict__ X, int64_t ldx,
                                                     double* __restrict__ R, int64_t ldr, int64_t m, int64_t n,
                                                     const unsigned long long* slot_a,
                                                     const unsigned long long* slot_b,
                                                     const unsigned long long* slot_x, unsigned long long* rmax,
                                                     const int* skip) {
  if (skip && ld_volatile(skip)) return;
  residual_df_tile(Ah, Al, lda, Bh, Bl, ldb, C, ldc, X, ldx, R, ldr, m, n, slot_a, slot_b, slot_x, rmax,
                   static_cast<int64_t>(blockIdx.x) * GT, static_cast<int64_t>(blockIdx.y) * GT);
}

// Float pair (hi, lo) of src * 2^-s, s from the larger of two max slots; quasi != 0
// keeps only r <= c+1.
__global__ void k_split_df(const double* __restrict__ src, int64_t lds, float* __restrict__ hi,
                           float* __restrict__ lo, int64_t ldd, int64_t rows, int64_t cols,
                           const unsigned long long* slot_a, const unsigned long long* slot_b, int quasi) {
  const unsigned long long a = *slot_a, b = slot_b ? *slot_b : 0ull;
  const int s = norm_exp(a > b ? slot_a : slot_b);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < rows * cols;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % rows, c = t / rows;
    const double v = (!quasi || r <= c + 1) ? mul2(src[r + c * lds], -s) : 0.0;
    const DF d = split_df(v);
    hi[r + c * ldd] = d.hi;
    lo[r + c * ldd] = d.lo;
  }
}

// max |X| over an m x n matrix (bit pattern slot).
__global__ void k_maxabs(const double* __restrict__ X, int64_t ldx, int64_t m, int64_t n, unsigned long long* out,
                         const int* skip) {
  if (skip && ld_volatile(skip)) return;
  double mx = 0.0;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < m * n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    mx = fmax(mx, fabs(X[(t % m) + (t / m) * ldx]));
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, mx);
}

}  // namespace sylv

namespace sylv {

// Batched gradient products (equation e = blockIdx.z): the same product and mask
// as k_grad_product, with per-equation operands.
struct GradDesc {
  const double* P;
  int64_t psi, psc;
  const double* Q;
  int64_t qsj, qsc;
  int64_t N, K;
  const double* T;
  int64_t ldt;
  double* D;
  int64_t ldd;
  double sign;      // -1 for dB of op(A) Y - Y op(B) = alpha C
  sylv_result* rs;  // the adjoint solve's record: D is multiplied by 2^-rs->log2scale
};

__global__ void __launch_bounds__(256) k_grad_product_batched(const GradDesc* __restrict__ gd) {
  const GradDesc g = gd[blockIdx.z];
  __shared__ __align__(16) double Ls[GK * GLD];
  __shared__ __align__(16) double Rs[GK * GLD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * GT, j0 = static_cast<int64_t>(blockIdx.y) * GT;
  if (i0 >= g.N || j0 >= g.N) return;
  const bool active = i0 <= j0 + GT;
  const int eu = unscale_exp(g.rs, 0);
  double acc[4][4] = {};
  if (active) {
    for (int64_t k0 = 0; k0 < g.K; k0 += GK) {
      for (int idx = tid; idx < GK * GT; idx += 256) {
        const int r = idx % GT, kk = idx / GT;
        const int64_t gi = i0 + r, gk = k0 + kk, gj = j0 + r;
        Ls[kk * GLD + r] = (gi < g.N && gk < g.K) ? g.P[gi * g.psi + gk * g.psc] : 0.0;
        Rs[kk * GLD + r] = (gj < g.N && gk < g.K) ? g.Q[gj * g.qsj + gk * g.qsc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ls[kk * GLD + tx * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Rs[kk * GLD + ty * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      if (r < g.N && c < g.N) {
        const bool keep = (r <= c) || (r == c + 1 && g.T[r + c * g.ldt] != 0.0);
        g.D[r + c * g.ldd] = keep ? unscale(g.sign * acc[i][j], eu, g.rs) : 0.0;
      }
    }
}

// Batched power-of-two scaling: M_e *= 2^(e_e - rs_e->log2scale) (equation e =
// blockIdx.y; rs null: 2^e_e).
struct ScaleDesc {
  double* M;
  int64_t ld, m, n;
  int64_t e;
  sylv_result* rs;
};
__global__ void k_scale_pow2_batched(const ScaleDesc* __restrict__ sd) {
  const ScaleDesc s = sd[blockIdx.y];
  const int eu = unscale_exp(s.rs, s.e);
  if (eu == 0) return;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < s.m * s.n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t % s.m, c = t / s.m;
    s.M[r + c * s.ld] = unscale(s.M[r + c * s.ld], eu, s.rs);
  }
}

}  // namespace sylv

namespace sylv {

// R <- R - (A D + D B) in binary32 arithmetic, for a correction D that is small
// compared to the solution: the products' rounding (~2^-24 |A| |D|) is far below
// the binary64-accurate residual the recurrence starts from.  A, B: the binary32
// parts of the scaled pair (AS = A 2^-sa); D (binary64) scaled by 2^-sd into binary32
// range; R_new = R - 2^(sa+sd) (AS DS + DS BS) with the final subtraction in
// binary64.  Records max |R_new|.  64 x 64 outputs per CTA, 4 x 4 per thread.
// One 64 x 64 output tile (rows i0.., columns j0..) of k_residual_update.
__device__ __forceinline__ void residual_update_tile(const float* __restrict__ Ah, int64_t lda,
                                                     const float* __restrict__ Bh, int64_t ldb,
                                                     const double* __restrict__ D, int64_t ldd,
                                                     double* __restrict__ R, int64_t ldr, int64_t m, int64_t n,
                                                     const unsigned long long* slot_a,
                                                     const unsigned long long* slot_b,
                                                     const unsigned long long* slot_d, unsigned long long* rmax,
                                                     int64_t i0, int64_t j0) {
  constexpr int LD = GT + 4;
  __shared__ __align__(16) float Ls[GK * LD], Rs[GK * LD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const unsigned long long ua = *slot_a, ub = *slot_b;
  const int sa = norm_exp(ua > ub ? slot_a : slot_b);
  const int sd = norm_exp(slot_d);
  float acc[4][4] = {};
  const int64_t ka = i0 > 0 ? i0 - 1 : 0;
  for (int64_t k0 = ka; k0 < m; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      Ls[kk * LD + r] = (gr < m && gk < m && gr <= gk + 1) ? Ah[gr + gk * lda] : 0.f;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      Rs[kk2 * LD + c] = (gk2 < m && gc < n) ? static_cast<float>(mul2(D[gk2 + gc * ldd], -sd)) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Ls[kk * LD + tx * 4 + i];
        b[i] = Rs[kk * LD + ty * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const int64_t kb_end = (j0 + GT + 1 < n) ? j0 + GT + 1 : n;
  for (int64_t k0 = 0; k0 < kb_end; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      const int r = idx % GT, kk = idx / GT;
      const int64_t gr = i0 + r, gk = k0 + kk;
      Ls[kk * LD + r] = (gr < m && gk < n) ? static_cast<float>(mul2(D[gr + gk * ldd], -sd)) : 0.f;
      const int kk2 = idx % GK, c = idx / GK;
      const int64_t gk2 = k0 + kk2, gc = j0 + c;
      Rs[kk2 * LD + c] = (gk2 < n && gc < n && gk2 <= gc + 1) ? Bh[gk2 + gc * ldb] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Ls[kk * LD + tx * 4 + i];
        b[i] = Rs[kk * LD + ty * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = j0 + ty * 4 + j;
      if (r < m && c < n) {
        const double v = R[r + c * ldr] - mul2(static_cast<double>(acc[i][j]), sa + sd);
        R[r + c * ldr] = v;
        mx = fmax(mx, fabs(v));
      }
    }
  mx = warp_max(mx);
  if ((tid & 31) == 0 && rmax) atomic_max_nonneg(rmax, mx);
}

__global__ void __launch_bounds__(256) k_residual_update(const float* __restrict__ Ah, int64_t lda,
                                                         const float* __restrict__ Bh, int64_t ldb,
                                                         const double* __restrict__ D, int64_t ldd,
                                                         double* __restrict__ R, int64_t ldr, int64_t m, int64_t n,
                                                         const unsigned long long* slot_a,
                                                         const unsigned long long* slot_b,
                                                         const unsigned long long* slot_d, unsigned long long* rmax,
                                                         const int* skip) {
  if (skip && ld_volatile(skip)) return;
  residual_update_tile(Ah, lda, Bh, ldb, D, ldd, R, ldr, m, n, slot_a, slot_b, slot_d, rmax,
                       static_cast<int64_t>(blockIdx.x) * GT, static_cast<int64_t>(blockIdx.y) * GT);
}

}  // namespace sylv
