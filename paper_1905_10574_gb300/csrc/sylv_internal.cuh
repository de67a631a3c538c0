// sylv_internal.cuh -- device-side data structures and helpers shared by the
// kernels of the GB300 triangular Sylvester solver (C ABI in include/sylv.h).
//
// Method: Schwarz & Kjelgaard Mikkelsen 2019, "Robust Task-Parallel Solution of
// the Triangular Sylvester Equation".  Tiles of Y are augmented tiles <alpha, X>
// (Sec. 2.2, Def. 1) whose scale alpha = 2^e is kept as an integer exponent e <= 0.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sylv.h"

namespace sylv {

constexpr int kThreads = 256;  // threads per CTA of every tile kernel

// Per-equation status bits (InstState::flags).
constexpr int kFlagNearSingular = 1;  // a small system's pivot was raised to smin
constexpr int kFlagNonfiniteOut = 2;  // a solved tile holds Inf/NaN (non-robust overflow)

// One equation of a (possibly batched) solve.  Element type of A, B, C is the
// kernel's T (double for the FP64 paths, float for the FP32 correction solves).
struct Inst {
  int64_t m, n;
  int64_t lda, ldb, ldc;
  const void* A;
  const void* B;
  void* C;
  int32_t t;           // nominal tile size
  int32_t pmax, qmax;  // capacity of the tile arrays (>= actual tile counts)
  int32_t robust;      // 1: Algorithm 4 with scaling; 0: no scaling (Algorithm 1 per tile)
  int32_t nob;         // 1: no B term, the robust triangular solve op(A) X = alpha C (B unused)
  int64_t rb, cb;      // offsets (ints) of the row/column tile boundaries in Work::ibuf
  int64_t tile;        // offset (elements) of this equation's per-tile arrays
  int64_t an, bn;      // offsets (doubles) of the tile-norm tables in Work::dbuf
  double omega;        // overflow threshold
  int64_t pk;          // first slot of this equation's packed tiles in Work::pack (see below)
};

// Per-equation results and bookkeeping, written by the kernels.
struct InstState {
  int32_t p, q;        // actual tile counts
  int32_t minexp;      // min over tiles of the local exponent (atomicMin)
  int32_t flags;       // kFlag* bits (atomicOr)
  int32_t err;         // first SYLV_ERR_* of this equation (atomicCAS from 0)
  int32_t nscale;      // scaling decisions taken (atomicAdd)
  unsigned long long amax, bmax;  // max |A|, |B| as binary64 bit patterns (atomicMax)
  double smin;         // pivot floor of the small solves
};

struct Task {
  int32_t inst;
  int32_t tile;  // k * qmax + l
};

struct Ctrl {
  int32_t ticket;   // next task of the persistent kernel
  int32_t workers;  // SM cap: CTAs of this launch inside the SM budget (reset with ticket)
  int32_t ntasks;   // tasks in Work::tasks
  int32_t err;      // first launch-wide error (timeout)
  int32_t nlevels;  // anti-diagonal levels in use
};

struct Work {
  Inst* inst;
  InstState* st;
  int32_t count;        // equations
  int32_t nlevels_max;  // capacity of the level arrays
  Task* tasks;
  Ctrl* ctrl;
  int32_t* lvl_cnt;
  int32_t* lvl_off;
  int32_t* lvl_cur;
  int32_t* ibuf;    // tile boundaries
  int32_t* texp;    // local exponent per tile
  // Ready word of each tile, 0 until the tile is final (release/acquire): bit 63 set,
  // bits 62..32 the high word of its infinity norm rounded up (an upper bound of the
  // norm with a 20-bit significand), bits 31..0 its exponent, so a consumer learns
  // readiness, exponent and norm bound from one load.
  unsigned long long* tflag;
  double* tnorm;    // infinity norm of each final tile (as stored, i.e. scaled)
  double* dbuf;     // off-diagonal tile norms of A and B
  sylv_result* res; // per-equation results
  const int* skip;  // if non-null and nonzero, the DAG kernel returns at once
  // Per-equation skip (batched refinement): if non-null, the tasks of equation e are
  // skipped (their tiles only marked final) while eqskip[e * eqskip_stride] != 0.
  const int* eqskip;
  int32_t eqskip_stride;
  double* fact;     // per-CTA store of factored small systems (fact_stride doubles each)
  int32_t* factp;   // per-CTA packed pivot data (TT*TT ints each)
  int64_t fact_stride;
  int32_t* smbusy;  // per SM: CTAs of this launch inside a diagonal-tile solve (1024 slots)
  int32_t prio;     // 1: update GEMMs yield the SM while a diagonal solve runs on it
  int64_t timeout_ns;
  int32_t max_tiles;  // max over equations of pmax * qmax
  int32_t sm_limit;   // > 0: CTAs (except CTA 0) on SMs with id >= sm_limit leave at once
  // Packed operand tiles (null: the kernel stages tiles from A, B, C directly).  One
  // slot holds a tile in the shared-memory operand layout of the update GEMM (TT rows
  // of k, row stride TT + 2, zero-padded), so one bulk copy stages it.  Per equation,
  // from slot pk: A_ki (pmax x pmax slots, left operand), B_jl (qmax x qmax, right
  // operand), then every final Y_kl twice (pmax x qmax each): as a left operand
  // (column-major) and as a right operand (row-major).
  char* pack;
  int64_t pack_slot;  // bytes per slot
};

// Slot numbers within an equation's packed region.
__host__ __device__ inline int64_t pack_a(const Inst& I, int k, int i) { return I.pk + static_cast<int64_t>(k) * I.pmax + i; }
__host__ __device__ inline int64_t pack_b(const Inst& I, int j, int l) {
  return I.pk + static_cast<int64_t>(I.pmax) * I.pmax + static_cast<int64_t>(j) * I.qmax + l;
}
__host__ __device__ inline int64_t pack_yl(const Inst& I, int k, int l) {
  return I.pk + static_cast<int64_t>(I.pmax) * I.pmax + static_cast<int64_t>(I.qmax) * I.qmax +
         static_cast<int64_t>(k) * I.qmax + l;
}
__host__ __device__ inline int64_t pack_yr(const Inst& I, int k, int l) {
  return pack_yl(I, k, l) + static_cast<int64_t>(I.pmax) * I.qmax;
}
__host__ __device__ inline int64_t pack_slots(int64_t pmax, int64_t qmax) { return (pmax + qmax) * (pmax + qmax); }

// ---------------------------------------------------------------- power-of-two scaling
// 2^e as binary64 for e in [-1022, 1023]: biased exponent e + 1023, zero fraction.
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
}
// 2^e as binary32 for e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// x * 2^e: exact whenever the result is a normal number (multiplication by a power
// of two only changes the exponent); very negative e is applied in normal-range steps.
__device__ __forceinline__ double mul2(double x, int e) {
  if (e == 0) return x;
  if (e < -2200) return x * 0.0;
  while (e < -1022) {
    x *= pow2d(-1022);
    e += 1022;
  }
  while (e > 1023) {
    x *= pow2d(1023);
    e -= 1023;
  }
  return x * pow2d(e);
}
__device__ __forceinline__ float mul2(float x, int e) {
  if (e == 0) return x;
  if (e < -400) return x * 0.0f;
  while (e < -126) {
    x *= pow2f(-126);
    e += 126;
  }
  while (e > 127) {
    x *= pow2f(127);
    e -= 127;
  }
  return x * pow2f(e);
}

// floor(log2 x) for finite x > 0, from the binary64 exponent field (subnormals via
// the position of the leading fraction bit).
__device__ __forceinline__ int floor_log2(double x) {
  const long long b = __double_as_longlong(x);
  const int be = static_cast<int>((b >> 52) & 0x7ff);
  if (be) return be - 1023;
  const long long frac = b & 0xFFFFFFFFFFFFFLL;
  return (63 - __clzll(frac)) - 1074;
}
// ceil(log2 x) for finite x > 0.
__device__ __forceinline__ int ceil_log2(double x) {
  const long long b = __double_as_longlong(x);
  const int be = static_cast<int>((b >> 52) & 0x7ff);
  const long long frac = b & 0xFFFFFFFFFFFFFLL;
  if (be) return frac ? be - 1022 : be - 1023;
  const int f = (63 - __clzll(frac)) - 1074;
  return (__popcll(frac) == 1) ? f : f + 1;
}

// x = f * 2^e with f in [1, 2), for finite x > 0: e from the exponent field
// (floor_log2), f by an exact power-of-two rescaling.
struct FracExp {
  double f;
  int e;
};
__device__ __forceinline__ FracExp frac_exp(double x) {
  const int e = floor_log2(x);
  return {mul2(x, -e), e};
}
// f * 2^d as an upper bound for f in [1, 4): exact while the result is normal;
// below that the bound 2^(d+2) is taken at 2^-998 (d < -1000).
__device__ __forceinline__ double shifted_up(double f, int d) { return d < -1000 ? 0x1p-998 : mul2(f, d); }

// ProtectUpdate (Sec. 2.1).  c, t, x are upper bounds of ||C||, ||A||, ||Y|| in
// [0, omega]; returns z <= 0 such that 2^z (c + t x) <= omega.  The test works on
// significands and exponents: with c = f_c 2^e_c, t = f_t 2^e_t, x = f_x 2^e_x and
// E = max(e_c, e_t + e_x),  c + t x = S 2^E  where S = f_c 2^(e_c-E) + f_t f_x 2^(e_t+e_x-E)
// lies in [1, 6).  So E + 3 <= log2 omega needs no scaling.  Otherwise S is bounded
// from above by arithmetic rounded towards +inf (S+ >= S), and with omega = f_w 2^e_w
// z = e_w - E + floor(log2(f_w / S+)), the quotient rounded towards -inf:
// 2^z S 2^E <= 2^e_w (f_w / S+) S <= omega.  z is the largest power of two the bound
// allows unless S+ rounds across a power of two (then it is one binade smaller).
__device__ __forceinline__ int protect_update(double c, double t, double x, double omega) {
  if (!(t > 0.0) || !(x > 0.0)) return 0;  // no update term: c <= omega already
  const FracExp ft = frac_exp(t), fx = frac_exp(x), fw = frac_exp(omega);
  const int ep = ft.e + fx.e;
  FracExp fc{0.0, ep};
  if (c > 0.0) fc = frac_exp(c);
  const int E = max(ep, fc.e);
  if (E + 3 <= fw.e) return 0;
  const double sp = shifted_up(__dmul_ru(ft.f, fx.f), ep - E);
  const double sc = c > 0.0 ? shifted_up(fc.f, fc.e - E) : 0.0;
  const double q = __ddiv_rd(fw.f, __dadd_ru(sc, sp));  // in (1/6, 2)
  return min(0, fw.e - E + floor_log2(q));
}

// ProtectDivision (Sec. 2.1) for |b| <= omega and divisor magnitude d > 0: returns
// the largest z <= 0 with 2^z |b| / d <= omega.  With |b| = f_b 2^e_b, d = f_d 2^e_d,
// omega = f_w 2^e_w the bound reads 2^z f_b 2^e_b <= f_d f_w 2^(e_d + e_w), so
// z = e_d + e_w - e_b + floor(log2(f_d f_w / f_b)), the ratio rounded towards -inf
// (then 2^z |b| <= d omega holds).  For a power-of-two omega the ratio f_d / f_b lies
// in (1/2, 2) and its floor(log2) survives the rounding, so z is exactly the largest.
__device__ __forceinline__ int protect_division(double b, double d, double omega) {
  b = fabs(b);
  d = fabs(d);
  if (!(b > 0.0) || d >= 1.0) return 0;  // |b| <= omega and d >= 1: |b| / d <= omega
  const FracExp fb = frac_exp(b), fd = frac_exp(d), fw = frac_exp(omega);
  const double r = __ddiv_rd(__dmul_rd(fd.f, fw.f), fb.f);  // in (1/2, 4)
  return min(0, fd.e + fw.e - fb.e + floor_log2(r));
}

// ---------------------------------------------------------------- inter-CTA signalling
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// The ready word of a final tile (see Work::tflag) and its two fields.
__device__ __forceinline__ unsigned long long tile_word(int e, double nrm) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(nrm)) & 0x7FFFFFFFFFFFFFFFull;
  unsigned long long hi = b >> 32;
  if ((b & 0xFFFFFFFFull) && hi < 0x7FF00000ull) ++hi;  // round the kept high word up
  return (1ull << 63) | ((hi & 0x7FFFFFFFull) << 32) | static_cast<uint32_t>(e);
}
__device__ __forceinline__ int word_exp(unsigned long long w) { return static_cast<int>(static_cast<uint32_t>(w)); }
__device__ __forceinline__ double word_norm(unsigned long long w) {
  return __longlong_as_double(static_cast<long long>(((w >> 32) & 0x7FFFFFFFull) << 32));
}

// Wait (thread-level) until *flag != 0.  Bounded: gives up after timeout_ns of
// global time or as soon as another CTA has recorded a launch-wide error, and
// then records SYLV_ERR_TIMEOUT (first error wins) and returns false.
__device__ __forceinline__ bool wait_flag(const int* flag, Ctrl* ctrl, long long timeout_ns) {
  if (ld_acquire(flag)) return true;
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  for (;;) {
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
    if (ld_acquire(flag)) return true;
    if (ld_volatile(&ctrl->err)) return false;
    if (static_cast<long long>(global_ns() - t0) > timeout_ns) {
      atomicCAS(&ctrl->err, 0, SYLV_ERR_TIMEOUT);
      return false;
    }
  }
}

// The same wait on a tile's 64-bit ready word; *word receives it.
__device__ __forceinline__ bool wait_word(const unsigned long long* flag, Ctrl* ctrl, long long timeout_ns,
                                          unsigned long long* word) {
  if ((*word = ld_acquire64(flag)) != 0) return true;
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  for (;;) {
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
    if ((*word = ld_acquire64(flag)) != 0) return true;
    if (ld_volatile(&ctrl->err)) return false;
    if (static_cast<long long>(global_ns() - t0) > timeout_ns) {
      atomicCAS(&ctrl->err, 0, SYLV_ERR_TIMEOUT);
      return false;
    }
  }
}

// Non-negative doubles order like their bit patterns (NaN above +Inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, static_cast<unsigned long long>(__double_as_longlong(v)));
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_min(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void set_err(InstState* st, int code) { atomicCAS(&st->err, 0, code); }

__device__ __forceinline__ unsigned sm_id() {
  unsigned id;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
  return id & 1023u;
}

}  // namespace sylv
