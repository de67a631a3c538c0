// sylv_dag.cuh -- the persistent tile-DAG kernel of the robust tiled solver
// (Algorithm 4 of Schwarz & Kjelgaard Mikkelsen 2019), templated on the tile
// capacity TT, the element type T and robust/non-robust mode.
//
// Work decomposition.  Tile (k,l) of Y (0-based, p x q tiles) depends on tiles
// (i,l), i > k, through Y_kl -= A_ki Y_il and on tiles (k,j), j < l, through
// Y_kl -= Y_kj B_jl (the block form of eqs. (6) and (8), with the index ranges that an
// upper-triangular A and B imply).  Instead of tasks with locks (Sec. 2.2), one
// CTA owns a tile from start to finish ("owner computes"): it pulls every
// incoming update in a fixed order (producers sorted by their anti-diagonal,
// which is the order in which they finish), then solves the diagonal problem
// A_kk Z + Z B_ll = beta Y_kl, stores Y_kl, its exponent and its norm, and
// publishes a ready flag (release).  Consumers wait on flags (acquire, bounded
// by a timeout).  Tasks are handed out by an atomic ticket in anti-diagonal
// order, so a CTA only ever waits for tiles whose tickets were taken earlier by
// running CTAs: no deadlock, whatever the grid size.  The accumulation order is
// fixed, so results are bitwise reproducible.
//
// Robust updates (Algorithm 3 with one operand a tile of A or B, scale 1): the
// accumulator carries exponent e_acc and a running upper bound nb of its
// infinity norm; for a producer with exponent e_p and exact norm y_p,
//   eta = min(e_acc, e_p)
//   zeta = ProtectUpdate(2^(eta-e_acc) nb, ||A_ki||, 2^(eta-e_p) y_p)   (or with
//          the roles of the last two swapped for Y_kj B_jl)
//   delta = eta + zeta;  acc <- 2^(delta-e_acc) acc - A_ki (2^(delta-e_p) Y_il).
// The printed Algorithm 3 applies delta to both factors of the product, which
// scales it by delta^2; with the A/B tile at scale 1 the product needs delta once.
#pragma once

#include <type_traits>

#include "sylv_internal.cuh"

namespace sylv {

// Merging of consecutive 1x1 blocks into pseudo 2x2 blocks in the diagonal solves
// (merge_blocks); a build may turn it off for comparison.
#ifndef SYLV_MERGE_DIAG
#define SYLV_MERGE_DIAG 1
#endif
// Left-looking diagonal solves (diag_solve's first phase); a build may turn it off
// for comparison, leaving the right-looking wavefront alone.
#ifndef SYLV_LEFT_DIAG
#define SYLV_LEFT_DIAG 1
#endif

template <int TT, typename T>
struct DagSmem {
  static constexpr int LDG = TT + 2;  // row stride of the GEMM operands (16-byte aligned rows)
  static constexpr int LDY = TT + 1;  // leading dimension of the Y, A_kk, B_ll tiles
  // Producers staged together in one GEMM pass: binary32 tiles are half the size,
  // and the FP32 correction solves are bound by per-update latency, so they stage more.
  static constexpr int G = sizeof(T) == 4 ? (TT <= 32 ? 6 : 2) : (TT <= 32 ? 3 : 1);
  T L[G * TT * LDG];                  // left GEMM operands, k-major; A_kk in the diagonal phases
  T R[G * TT * LDG];                  // right GEMM operands, k-major; B_ll in the diagonal phases
  int gside[G], gprod[G], gk[G], goff[G];  // the current group of producers
  int gsop[G];                        // per producer: power of two its Y operand takes (scaled group)
  int gn, gktot, gfast;
  // The binary32 tile-32 kernel's group product: the four k-interleaved partial tiles
  // (see gemm_sub_split4), column-major 32 x 32 each.
  static constexpr bool kSplitK = sizeof(T) == 4 && TT == 32;
  alignas(16) T kred[kSplitK ? 4 * TT * TT : 1];
  T Y[TT * LDY];                      // the tile being solved (column-major)
  // Small-system inverses in shared memory for tile capacity 32; the tile-64 kernels
  // keep them in the CTA's global slot.
  static constexpr bool kFactSmem = (TT <= 32);
  // The stored inverses are kept in the tile's precision: the binary32 kernel solves
  // its small systems in binary32 (its corrections are refined in binary64 anyway).
  using FactT = typename std::conditional<kFactSmem, T, double>::type;
  FactT fact[kFactSmem ? 5 * TT * TT : 1];       // inverse store (see pair_offset), if kFactSmem
  int factp[kFactSmem ? TT * TT : 1];            // per pair: bit 16 = a pivot was raised, if kFactSmem
  unsigned short eord[TT * TT];       // tile elements in wavefront order: row | col << 6 | vec index << 12
  short sstart[2 * TT];               // first entry of each wavefront step in eord
  unsigned long long acolmax[TT];     // per A block kb: max_r<start(kb) sum_i in kb |A[r,i]| (bits)
  unsigned long long bcolmax[TT];     // per B block lb: max_c>=end(lb) sum_j in lb |B[j,c]| (bits)
  short pr0[TT], pma[TT];             // this step: first row and height of the block solved in column block lb
  unsigned wmax[kThreads / 32];       // per-warp bound on |y| over unsolved elements (high word, rounded up)
  unsigned wz[2][kThreads / 32];      // left-looking phase: per-warp bound on |z| of a step (by step parity)
  int pe[TT];                         // scale exponent of each solved block of this step
  int pa[TT + 1];                     // factor-store offset of block row kb (see pair_offset)
  int qb2[TT + 1];                    // prefix sums of squared B block sizes
  short rowblk[TT], colblk[TT];       // block index of every row / column of the tile
  short astart[TT + 1], bstart[TT + 1];
  short aord[TT], bord[TT];           // blocks grouped by kind for the pair preparation (order_blocks)
  int acnt[3], bcnt[3];               // blocks of each kind: merged pseudo, 2x2, 1x1
  unsigned long long apsd, bpsd;      // diagonal solve: blocks that are two merged 1x1 blocks (bit per block)
  unsigned long long umax;
  unsigned long long stage_bar;        // mbarrier of the bulk-copy staging (packed tiles)
  double nb_acc;
  int task, abort, e_acc, sacc, sop, g, e_diag, pb, qb, nscale, flags, slow, skipt;
};

// Upper bound on log2|v| for finite v (exponent field + 1; 2^-1022 for zero/subnormals).
__device__ __forceinline__ int ub_log2(double v) {
  return static_cast<int>((__double_as_longlong(v) >> 52) & 0x7ff) - 1022;
}
// The same for binary32 (2^-126 for zero/subnormals; 129 for infinities and NaNs).
__device__ __forceinline__ int ub_log2(float v) { return static_cast<int>((__float_as_uint(v) >> 23) & 0xff) - 126; }
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}
// x + y, rounded upwards in binary32 (sums that must bound a norm from above); plain
// binary64 addition otherwise.
__device__ __forceinline__ double add_up(double x, double y) { return x + y; }
__device__ __forceinline__ float add_up(float x, float y) { return __fadd_ru(x, y); }
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Shared-memory address, bulk copy global -> shared completing on an mbarrier, and a
// bounded wait on an mbarrier phase (false on timeout or when a CTA recorded an error).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
template <typename T>
__device__ __forceinline__ void bulk_copy_g2s(T* dst, const char* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, const Ctrl* ctrl,
                                                  long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63) {
      if (ld_volatile(&ctrl->err)) return false;
      if (static_cast<long long>(global_ns() - t0) > timeout_ns) return false;
    }
  }
}

// ProtectUpdate with an integer fast path: when c + t x < 2^e_omega is evident from
// the exponent fields alone (eo = floor(log2 omega)), no FP64 arithmetic runs.
__device__ __forceinline__ int guard_update(double c, double t, double x, double omega, int eo) {
  const int bnd = max(ub_log2(c), ub_log2(t) + ub_log2(x)) + 1;
  if (bnd <= eo) return 0;
  return protect_update(fabs(c), fabs(t), fabs(x), omega);
}
// ProtectDivision for z = r * rcp with rcp = 1/d, integer fast path first.
__device__ __forceinline__ int guard_division(double r, double d, double rcp, double omega, int eo) {
  if (ub_log2(r) + ub_log2(rcp) <= eo) return 0;
  return protect_division(r, d, omega);
}

// ----------------------------------------------------------------------------
// Small Sylvester systems (Sec. 2.1): A11 Z + Z B11 = beta R with A11 ma x ma,
// B11 nb x nb (ma, nb in {1,2}) is (I (x) A11 + B11^T (x) I) vec Z = beta vec R, an
// s x s system M vec Z = beta vec R (s = ma nb).  The matrix does not depend on the
// right-hand side, so each tile factors it once per pair (Gaussian elimination
// with complete pivoting, pivots below smin raised to smin) and stores its inverse
// (pair_prepare).  In the common case a wavefront step then computes
// every element of Z as one dot product, z_e = sum_u Minv[e][u] r_u, one thread per
// element; that is safe from overflow whenever ||Minv||_inf max|r| stays below
// omega by a margin (an exponent test).  Otherwise the block is solved by
// pair_solve_guarded: the same eliminations applied to the right-hand side, each
// update guarded by ProtectUpdate and each division (a multiplication by the stored
// reciprocal) by ProtectDivision, as the robust small solve of Algorithm 2 requires.
// pair_factor's layout: multipliers below the diagonal, U on and above it, 1/pivot
// after the s*s entries; the row/column interchanges in a packed int (2 bits each;
// bit 16: a pivot was raised).
// A pseudo block (two 1x1 blocks merged, psa / psb) makes the system block
// triangular: with level(i, j) = (psa ? 1 - i : 0) + (psb ? j : 0), an element
// depends only on elements of lower levels (the bottom row of a pseudo A block and
// the left column of a pseudo B block come first).  The pivots are searched within
// the lowest level not yet eliminated, so that no interchange mixes levels: the
// factors keep the structure's exact zeros and the solve is the substitution of the
// 1x1 and 2x2 parts one after another (each part's pivots are those it has alone).
// Complete pivoting over the whole system would instead pivot on a large coupling
// entry and lose the small elements of the block (componentwise), which the
// substitution of Algorithm 2 over the unmerged blocks keeps.
__device__ inline int pair_factor(int ma, int nb, bool psa, bool psb, const double* a, const double* b, double smin,
                                  double* out) {
  const int s = ma * nb;
  double M[4][4];
  int pack = 0;
  int rlev[4], clev[4];  // level of the equation in row position u / unknown in column v
  for (int u = 0; u < s; ++u) {
    const int i = u % ma, j = u / ma;
    rlev[u] = clev[u] = (psa ? 1 - i : 0) + (psb ? j : 0);
    for (int v = 0; v < s; ++v) {
      const int i2 = v % ma, j2 = v / ma;
      double e = 0.0;
      if (j == j2) e += a[i + 2 * i2];
      if (i == i2) e += b[j2 + 2 * j];
      M[u][v] = e;
    }
  }
  int cperm[4] = {0, 1, 2, 3};
  for (int st = 0; st < s; ++st) {
    int lev = 3;
    for (int u = st; u < s; ++u) lev = min(lev, rlev[u]);
    int pr = st, pc = st;
    unsigned long long best = 0;
    bool first = true;
    for (int u = st; u < s; ++u)
      for (int v = st; v < s; ++v) {
        if (rlev[u] != lev || clev[v] != lev) continue;
        const unsigned long long mag = abs_bits(M[u][v]);
        if (first || mag > best) {
          best = mag;
          pr = u;
          pc = v;
          first = false;
        }
      }
    if (pr != st) {
      for (int v = 0; v < s; ++v) {
        const double tmp = M[st][v];
        M[st][v] = M[pr][v];
        M[pr][v] = tmp;
      }
      const int lt = rlev[st];
      rlev[st] = rlev[pr];
      rlev[pr] = lt;
    }
    if (pc != st) {
      for (int u = 0; u < s; ++u) {
        const double tmp = M[u][st];
        M[u][st] = M[u][pc];
        M[u][pc] = tmp;
      }
      const int lt = clev[st];
      clev[st] = clev[pc];
      clev[pc] = lt;
    }
    const int ct = cperm[st];
    cperm[st] = cperm[pc];
    cperm[pc] = ct;
    pack |= (pr & 3) << (2 * st);
    if (fabs(M[st][st]) < smin) {
      M[st][st] = smin;
      pack |= 1 << 16;
    }
    const double rcp = 1.0 / M[st][st];
    out[s * s + st] = rcp;
    for (int u = st + 1; u < s; ++u) {
      const double l = M[u][st] * rcp;
      M[u][st] = l;
      for (int v = st + 1; v < s; ++v) M[u][v] = fma(-l, M[st][v], M[u][v]);
    }
  }
  for (int u = 0; u < s; ++u) pack |= (cperm[u] & 3) << (8 + 2 * u);
  for (int u = 0; u < s; ++u)
    for (int v = 0; v < s; ++v) out[u * s + v] = M[u][v];
  return pack;
}

// Right-hand side of a factored pair of size S (1, 2 or 4): r (vec order) in, Z out.
// Returns log2(beta).  Compile-time S keeps r in registers (interchanges by selects).
template <int S>
__device__ __noinline__ int pair_solve_guarded(const double* f, int pack, double (&r)[4], double omega, int eo,
                                               bool robust) {
  int lb = 0;
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const int pr = (pack >> (2 * st)) & 3;
#pragma unroll
    for (int k = st + 1; k < S; ++k)
      if (pr == k) {
        const double tmp = r[st];
        r[st] = r[k];
        r[k] = tmp;
      }
  }
#pragma unroll
  for (int st = 0; st < S; ++st)
#pragma unroll
    for (int u = st + 1; u < S; ++u) {
      const double l = f[u * S + st];
      if (robust) {
        const int z = guard_update(r[u], l, r[st], omega, eo);
        if (z) {
#pragma unroll
          for (int w = 0; w < S; ++w) r[w] = mul2(r[w], z);
          lb += z;
        }
      }
      r[u] = fma(-l, r[st], r[u]);
    }
#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
#pragma unroll
    for (int v = i + 1; v < S; ++v) {
      const double uiv = f[i * S + v];
      if (robust) {
        const int z = guard_update(r[i], uiv, r[v], omega, eo);
        if (z) {
#pragma unroll
          for (int w = 0; w < S; ++w) r[w] = mul2(r[w], z);
          lb += z;
        }
      }
      r[i] = fma(-uiv, r[v], r[i]);
    }
    const double rcp = f[S * S + i];
    if (robust) {
      const int z = guard_division(r[i], f[i * S + i], rcp, omega, eo);
      if (z) {
#pragma unroll
        for (int w = 0; w < S; ++w) r[w] = mul2(r[w], z);
        lb += z;
      }
    }
    r[i] = r[i] * rcp;
  }
  double x[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < S; ++u) {
    const int cu = (pack >> (8 + 2 * u)) & 3;
#pragma unroll
    for (int t = 0; t < S; ++t)
      if (cu == t) x[t] = r[u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) r[u] = x[u];
  return lb;
}

// Magnitude bits (for pivot search) and limits of the small-system compute type.
__device__ __forceinline__ unsigned long long mag_bits(double v) { return abs_bits(v); }
__device__ __forceinline__ unsigned mag_bits(float v) { return __float_as_uint(v) & 0x7fffffffu; }
template <typename CT>
struct Lim;
template <>
struct Lim<double> {
  static __device__ __forceinline__ double big() { return 1.7976931348623157e308; }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};
template <>
struct Lim<float> {
  static __device__ __forceinline__ float big() { return 3.4028234663852886e38f; }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

// ||Minv||_inf <= s max |m_eu| (a row holds s entries): the bound the solves' bound
// test needs, from the entries' bit patterns (binary64 row sums would cost about s^2
// instructions on the 1/64-rate FP64 pipe); infinite when an entry is not finite.
template <typename CT>
struct MagT;
template <>
struct MagT<double> {
  using B = unsigned long long;
  static constexpr B kInf = 0x7FF0000000000000ull;
  static __device__ __forceinline__ double val(B b) { return __longlong_as_double(static_cast<long long>(b)); }
};
template <>
struct MagT<float> {
  using B = unsigned;
  static constexpr B kInf = 0x7F800000u;
  static __device__ __forceinline__ float val(B b) { return __uint_as_float(b); }
};
template <typename CT>
__device__ __forceinline__ CT inv_norm_bound(typename MagT<CT>::B mb, int s) {
  return mb >= MagT<CT>::kInf ? Lim<CT>::inf() : MagT<CT>::val(mb) * static_cast<CT>(s);
}

// The factorization of pair_factor for a compile-time block shape (MA x MA with
// NB x NB), in registers, followed by the inverse: column k of Minv solves
// M x = e_k with the same interchanges, multipliers and reciprocals.  Writes Minv
// row-major (Minv[e][u] at out[e*S+u]) and ||Minv||_inf at out[S*S]; a non-finite
// entry (a raised pivot of a near-singular pair can overflow) stores an infinite
// norm, which sends every solve of the pair to the guarded path.  Returns the
// packed interchanges.
template <int MA, int NB, typename CT = double>
__device__ __forceinline__ int pair_prepare(const CT (&a)[4], const CT (&b)[4], double smin, CT* out) {
  constexpr int S = MA * NB;
  const CT sm = static_cast<CT>(smin);
  CT M[S][S];
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int v = 0; v < S; ++v) {
      CT e = -CT(0);  // -0 + x folds to x: only the diagonal entries take an addition
      if (u / MA == v / MA) e += a[(u % MA) + 2 * (v % MA)];
      if (u % MA == v % MA) e += b[(v / MA) + 2 * (u / MA)];
      M[u][v] = e;
    }
  int cperm[S];
#pragma unroll
  for (int u = 0; u < S; ++u) cperm[u] = u;
  CT rcp[S];
  int pack = 0;
#pragma unroll
  for (int st = 0; st < S; ++st) {
    int pr = st, pc = st;
    auto best = mag_bits(M[st][st]);
#pragma unroll
    for (int u = st; u < S; ++u)
#pragma unroll
      for (int v = st; v < S; ++v) {
        const auto mg = mag_bits(M[u][v]);
        if (mg > best) {
          best = mg;
          pr = u;
          pc = v;
        }
      }
#pragma unroll
    for (int k = st + 1; k < S; ++k)
      if (pr == k)
#pragma unroll
        for (int v = 0; v < S; ++v) {
          const CT t = M[st][v];
          M[st][v] = M[k][v];
          M[k][v] = t;
        }
#pragma unroll
    for (int k = st + 1; k < S; ++k)
      if (pc == k) {
#pragma unroll
        for (int u = 0; u < S; ++u) {
          const CT t = M[u][st];
          M[u][st] = M[u][k];
          M[u][k] = t;
        }
        const int ct = cperm[st];
        cperm[st] = cperm[k];
        cperm[k] = ct;
      }
    pack |= (pr & 3) << (2 * st);
    if (fabs(M[st][st]) < sm) {
      M[st][st] = sm;
      pack |= 1 << 16;
    }
    rcp[st] = CT(1) / M[st][st];
#pragma unroll
    for (int u = st + 1; u < S; ++u) {
      const CT l = M[u][st] * rcp[st];
      M[u][st] = l;
#pragma unroll
      for (int v = st + 1; v < S; ++v) M[u][v] = fma(-l, M[st][v], M[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < S; ++u) pack |= (cperm[u] & 3) << (8 + 2 * u);
  CT inv[S][S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    CT r[S];
#pragma unroll
    for (int u = 0; u < S; ++u) r[u] = (u == k) ? CT(1) : CT(0);
#pragma unroll
    for (int st = 0; st < S; ++st) {
      const int pr = (pack >> (2 * st)) & 3;
#pragma unroll
      for (int kk = st + 1; kk < S; ++kk)
        if (pr == kk) {
          const CT t = r[st];
          r[st] = r[kk];
          r[kk] = t;
        }
    }
#pragma unroll
    for (int st = 0; st < S; ++st)
#pragma unroll
      for (int u = st + 1; u < S; ++u) r[u] = fma(-M[u][st], r[st], r[u]);
#pragma unroll
    for (int i = S - 1; i >= 0; --i) {
#pragma unroll
      for (int v = i + 1; v < S; ++v) r[i] = fma(-M[i][v], r[v], r[i]);
      r[i] = r[i] * rcp[i];
    }
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t)
        if (cperm[u] == t) inv[t][k] = r[u];
  }
  typename MagT<CT>::B mb = 0;
#pragma unroll
  for (int e = 0; e < S; ++e)
#pragma unroll
    for (int u = 0; u < S; ++u) {
      out[e * S + u] = inv[e][u];
      mb = max(mb, mag_bits(inv[e][u]));
    }
  out[S * S] = inv_norm_bound<CT>(mb, S);
  return pack;
}

// Upper bound of |v| kept in 32 bits: the high word of its bit pattern, plus one
// unless the low word is zero (so the bound never falls below |v|).
__device__ __forceinline__ unsigned hi_bound(double v) {
  const unsigned long long b = abs_bits(v);
  return static_cast<unsigned>(b >> 32) + ((b & 0xffffffffull) != 0ull ? 1u : 0u);
}
// The same bound for a binary32 value from its bit pattern alone (no FP64 instruction,
// which would occupy the 1/64-rate FP64 pipe): the double's high word is the float's
// exponent rebiased and its mantissa's top 20 bits, plus one when the 3 low mantissa
// bits (the double's low word) are nonzero.  Subnormal floats are bounded by 2^-126,
// infinities and NaNs map to the infinite bound.
__device__ __forceinline__ unsigned hi_bound(float v) {
  const unsigned b = __float_as_uint(v) & 0x7fffffffu;
  const unsigned e = b >> 23, m = b & 0x7fffffu;
  if (e == 0) return m ? ((1023u - 126u) << 20) : 0u;
  if (e == 255) return 0x7ff00000u;
  return ((e + 896u) << 20) + (m >> 3) + ((m & 7u) ? 1u : 0u);
}
// Exact binary32 -> binary64 conversion by rebiasing the bit pattern (normal values;
// zeros, subnormals, infinities and NaNs take the conversion instruction).
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0 || e == 255) return static_cast<double>(v);
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                                                     (static_cast<unsigned long long>(e + 896u) << 52) |
                                                     (static_cast<unsigned long long>(b & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double from_hi_bound(unsigned h) {
  return bits_to_double(static_cast<unsigned long long>(h) << 32);
}

// Block structure of an upper quasi-triangular tile (Sec. 1, eq. (4)): a nonzero
// M[i+1,i] starts a 2x2 block at i.  One warp; writes blk[i] (block of row i),
// start[b] (first row of block b, start[nblk] = N) and returns nblk.
template <typename T, int LD>
__device__ inline int scan_blocks(const T* M, int N, short* blk, short* start, int lane) {
  unsigned carry = 0;
  int count = 0;
  for (int base = 0; base < N; base += 32) {
    const int i = base + lane;
    const bool ps = (i + 1 < N) && (M[(i + 1) + i * LD] != T(0));
    const unsigned P = __ballot_sync(0xffffffffu, ps);
    const unsigned prevP = (P << 1) | carry;
    const bool st = (i < N) && !((prevP >> lane) & 1u);
    const unsigned S = __ballot_sync(0xffffffffu, st);
    const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
    const int idx = count + __popc(S & upto) - 1;
    if (i < N) blk[i] = static_cast<short>(idx);
    if (st) start[idx] = static_cast<short>(i);
    count += __popc(S);
    carry = (P >> 31) & 1u;
  }
  if (lane == 0) start[count] = static_cast<short>(N);
  return count;
}

// Pseudo blocks for the diagonal-tile solve: consecutive 1x1
// blocks are merged in pairs, so that the wavefront over the tile's blocks takes about
// half as many steps (each a chain of dependent FP64 operations and block barriers).
// A merged pair is solved as one small system whose inverse is composed from the
// inverses of its parts (pair_quad_prepare, pair_half_prepare), so a near-singular
// part raises exactly the pivot it raises on its own.  One warp, nblk <= 32; rewrites blk and
// start in place, returns the new count and sets *pseudo (bit per new block).
__device__ inline int merge_blocks(short* blk, short* start, int n, int nblk, unsigned long long* pseudo, int lane) {
  const int b = lane;
  const bool valid = b < nblk;
  const int sz = valid ? start[b + 1] - start[b] : 0;
  const short my_start = valid ? start[b] : short(0);
  const unsigned O = __ballot_sync(0xffffffffu, valid && sz == 1);
  const unsigned zeros_below = ~O & ((1u << b) - 1u);
  const int run0 = zeros_below ? 32 - __clz(zeros_below) : 0;  // first block of this run of 1x1 blocks
  const bool one = (O >> b) & 1u;
  const bool odd = ((b - run0) & 1) != 0;
  const bool head = one && !odd && b < 31 && ((O >> (b + 1)) & 1u);  // merges with block b+1
  const bool tail = one && odd;                                        // merged into block b-1
  const unsigned S = __ballot_sync(0xffffffffu, valid && !tail);       // blocks that start a new block
  const int nidx = __popc(S & (b == 31 ? 0xffffffffu : ((2u << b) - 1u))) - 1;
  const unsigned pm = __reduce_or_sync(0xffffffffu, head ? (1u << nidx) : 0u);
  __syncwarp();
  if (valid && !tail) start[nidx] = my_start;
  for (int i = lane; i < n; i += 32) {
    const int ob = blk[i];
    blk[i] = static_cast<short>(__popc(S & (ob == 31 ? 0xffffffffu : ((2u << ob) - 1u))) - 1);
  }
  const int count = __popc(S);
  if (lane == 0) {
    start[count] = static_cast<short>(n);
    *pseudo = pm;
  }
  __syncwarp();
  return count;
}

// The same merge for up to 64 blocks (tile capacity 64): lane 0 walks the blocks (a
// run of 1x1 blocks pairs from its first block, as above) compacting start in place,
// then the warp renumbers the rows.
__device__ inline int merge_blocks_long(short* blk, short* start, int n, int nblk, unsigned long long* pseudo,
                                        int lane) {
  int count = 0;
  if (lane == 0) {
    unsigned long long pm = 0;
    for (int b = 0; b < nblk;) {
      const short s0 = start[b];
      const bool pair = start[b + 1] - s0 == 1 && b + 1 < nblk && start[b + 2] - start[b + 1] == 1;
      start[count] = s0;  // count <= b: the entries still to be read lie above it
      if (pair) pm |= 1ull << count;
      b += pair ? 2 : 1;
      ++count;
    }
    start[count] = static_cast<short>(n);
    *pseudo = pm;
  }
  count = __shfl_sync(0xffffffffu, count, 0);
  __syncwarp();
  for (int i = lane; i < n; i += 32) {  // the last block starting at or before row i
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    blk[i] = static_cast<short>(lo);
  }
  __syncwarp();
  return count;
}

// A merged pair of two pseudo blocks (four 1x1 parts): the composed inverse in closed
// form.  With the parts' reciprocals i_ij = 1/d_ij, d_ij = a_ii + b_jj raised to smin
// like a 1x1 pair's pivot, and the couplings a12 = A[r0, r0+1], b12 = B[c0, c0+1],
// the solve order z10, z00, z11, z01 gives (vec order u = i + 2j)
//   z00 = i00 (r00 - a12 z10),  z10 = i10 r10,  z11 = i11 (r11 - b12 z10),
//   z01 = i01 (r01 - a12 z11 - b12 z00).
// Writes Minv row-major and ||Minv||_inf (infinity if not finite) in OutT; returns
// bit 16 if a part raised its pivot.
template <typename CT>
__device__ __forceinline__ int pair_quad_prepare(const CT (&a)[4], const CT (&b)[4], double smin, CT* out) {
  int flag = 0;
  const CT sm = static_cast<CT>(smin);
  auto inv = [&](CT d) {
    if (fabs(d) < sm) {
      d = sm;
      flag = 1 << 16;
    }
    return CT(1) / d;
  };
  const CT i00 = inv(a[0] + b[0]), i10 = inv(a[3] + b[0]), i01 = inv(a[0] + b[3]), i11 = inv(a[3] + b[3]);
  const CT a12 = a[2], b12 = b[2];
  const CT m[16] = {i00,
                        -a12 * i00 * i10,
                        CT(0),
                        CT(0),
                        CT(0),
                        i10,
                        CT(0),
                        CT(0),
                        -b12 * i01 * i00,
                        a12 * b12 * i01 * i10 * (i00 + i11),
                        i01,
                        -a12 * i01 * i11,
                        CT(0),
                        -b12 * i11 * i10,
                        CT(0),
                        i11};
  typename MagT<CT>::B mb = 0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    out[e] = m[e];
    mb = max(mb, mag_bits(m[e]));
  }
  out[16] = inv_norm_bound<CT>(mb, 4);
  return flag;
}

// A merged pair with one pseudo side, composed inline from its two parts' inverses
// (pair_prepare of each part, so a part raises exactly the pivots it raises alone).
// Pseudo A (rows split, bottom part solved first): Minv = [[It, -a12 It Ib], [0, Ib]]
// over (top, bottom) rows; pseudo B (columns split, left first):
// Minv = [[Il, 0], [-b12 Ir Il, Ir]] over (left, right) columns.  Each part has the
// other side's whole block (1x1 or 2x2).  Same output layout as pair_prepare.
template <typename CT>
__device__ __noinline__ int pair_half_prepare(int ma, int nb, bool pa, CT a0_, CT a1_, CT a2_, CT a3_, CT b0_, CT b1_,
                                              CT b2_, CT b3_, double smin, CT* out) {
  // The blocks' entries arrive as scalars, so the caller's arrays stay in registers.
  const CT a[4] = {a0_, a1_, a2_, a3_}, b[4] = {b0_, b1_, b2_, b3_};
  const int s = ma * nb;
  const int h = pa ? nb : ma;  // size of each part's system (the other side's block)
  CT P0[5], P1[5];              // part inverses (<= 2 x 2, row-major) and norms
  CT a0[4] = {CT(0), CT(0), CT(0), CT(0)}, a1[4] = {CT(0), CT(0), CT(0), CT(0)};
  CT b0[4] = {CT(0), CT(0), CT(0), CT(0)}, b1[4] = {CT(0), CT(0), CT(0), CT(0)};
  int flags;
  if (pa) {  // part 0: top row (a00), part 1: bottom row (a11); both with B
    a0[0] = a[0];
    a1[0] = a[3];
    flags = (h == 1) ? (pair_prepare<1, 1, CT>(a0, b, smin, P0) | pair_prepare<1, 1, CT>(a1, b, smin, P1))
                     : (pair_prepare<1, 2, CT>(a0, b, smin, P0) | pair_prepare<1, 2, CT>(a1, b, smin, P1));
  } else {  // part 0: left column (b00), part 1: right column (b11); both with A
    b0[0] = b[0];
    b1[0] = b[3];
    flags = (h == 1) ? (pair_prepare<1, 1, CT>(a, b0, smin, P0) | pair_prepare<1, 1, CT>(a, b1, smin, P1))
                     : (pair_prepare<2, 1, CT>(a, b0, smin, P0) | pair_prepare<2, 1, CT>(a, b1, smin, P1));
  }
  // Coupled block: pseudo A: top += -a12 It Ib (rows of the top part, columns of the
  // bottom part); pseudo B: right += -b12 Ir Il.
  const CT cpl = pa ? a[2] : b[2];
  CT m[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int u = 0; u < 4; ++u) m[e][u] = CT(0);
  // vec index of part p, local index t: pseudo A: element (i = p, j = t) -> p + 2t;
  // pseudo B: element (i = t, j = p) -> t + ma p.
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      if (t >= h || v >= h) continue;
      const int e0 = pa ? 0 + 2 * t : t, u0 = pa ? 0 + 2 * v : v;            // part 0
      const int e1 = pa ? 1 + 2 * t : t + ma, u1 = pa ? 1 + 2 * v : v + ma;  // part 1
      m[e0][u0] = P0[t * h + v];
      m[e1][u1] = P1[t * h + v];
      CT c = CT(0);  // (P_first_solved_after * P_solved_first)[t][v]
#pragma unroll
      for (int w = 0; w < 2; ++w)
        if (w < h) c = fma(pa ? P0[t * h + w] : P1[t * h + w], pa ? P1[w * h + v] : P0[w * h + v], c);
      if (pa)
        m[e0][u1] = -cpl * c;  // top row element from the bottom right-hand side
      else
        m[e1][u0] = -cpl * c;  // right column element from the left right-hand side
    }
  typename MagT<CT>::B mb = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e >= s) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (u >= s) continue;
      out[e * s + u] = m[e][u];
      mb = max(mb, mag_bits(m[e][u]));
    }
  }
  out[s * s] = inv_norm_bound<CT>(mb, s);
  return flags & (1 << 16);
}

// Blocks grouped by kind for the pair preparation: merged pseudo blocks first, then
// 2x2 blocks, then 1x1 blocks (stable within a kind).  The small systems of different
// kinds take different code, so a warp whose pairs mix kinds executes every kind's
// code in turn, which on the 1/64-rate FP64 pipe costs as much as the updates of
// several producers; with pairs enumerated kind by kind a warp mostly runs one.  One
// warp; writes ord[0..nblk) and cnt[3].
__device__ inline void order_blocks(const short* start, int nblk, unsigned long long pseudo, short* ord, int* cnt,
                                    int lane) {
  int n[3] = {0, 0, 0};
  for (int b0 = 0; b0 < nblk; b0 += 32) {
    const int b = b0 + lane;
    const bool v = b < nblk;
    const bool ps = v && b < 64 && ((pseudo >> b) & 1ull);
    const int kind = !v ? 3 : ps ? 0 : (start[b + 1] - start[b] == 2 ? 1 : 2);
#pragma unroll
    for (int t = 0; t < 3; ++t) n[t] += __popc(__ballot_sync(0xffffffffu, kind == t));
  }
  int off[3] = {0, n[0], n[0] + n[1]};
  const unsigned below = (1u << lane) - 1u;
  for (int b0 = 0; b0 < nblk; b0 += 32) {
    const int b = b0 + lane;
    const bool v = b < nblk;
    const bool ps = v && b < 64 && ((pseudo >> b) & 1ull);
    const int kind = !v ? 3 : ps ? 0 : (start[b + 1] - start[b] == 2 ? 1 : 2);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const unsigned m = __ballot_sync(0xffffffffu, kind == t);
      if (kind == t) ord[off[t] + __popc(m & below)] = static_cast<short>(b);
      off[t] += __popc(m);
    }
  }
  if (lane < 3) cnt[lane] = n[lane];
}

// Offset of pair (kb, lb) in the factor store: pairs are stored block row by block
// row, each taking s^2 + s doubles (s = ma nb).
template <int TT, typename T>
__device__ __forceinline__ int pair_offset(const DagSmem<TT, T>& sh, int kb, int lb, int ma) {
  return sh.pa[kb] + ma * ma * sh.qb2[lb] + ma * sh.bstart[lb];
}

// Diagonal-tile preparation, independent of Y: load A_kk into L and B_ll into R,
// find their 1x1/2x2 blocks, the norms the in-tile guards need, and factor every
// pair's small system into the CTA's factor store.  Runs right after a CTA takes a
// tile, while the tile's producers may still be running.
template <int TT, typename T, bool ROBUST>
__device__ void diag_prepare(DagSmem<TT, T>& sh, const T* A, int64_t lda, const T* B, int64_t ldb, int r0, int c0,
                             int mt, int nt, double smin, double* gfact, int* gfactp) {
  constexpr int LDY = DagSmem<TT, T>::LDY;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  using FactT = typename DagSmem<TT, T>::FactT;
  FactT* fact;
  int* factp;
  if constexpr (DagSmem<TT, T>::kFactSmem) {
    fact = sh.fact;
    factp = sh.factp;
  } else {
    fact = gfact;
    factp = gfactp;
  }
  T* Ak = sh.L;
  T* Bk = sh.R;
  for (int idx = tid; idx < TT * TT; idx += kThreads) {
    const int r = idx % TT, c = idx / TT;
    Ak[r + c * LDY] = (r < mt && c < mt && r <= c + 1) ? __ldg(&A[(r0 + r) + static_cast<int64_t>(r0 + c) * lda]) : T(0);
    Bk[r + c * LDY] = (B && r < nt && c < nt && r <= c + 1) ? __ldg(&B[(c0 + r) + static_cast<int64_t>(c0 + c) * ldb])
                                                             : T(0);
  }
  for (int i = tid; i < TT; i += kThreads) {
    sh.acolmax[i] = 0ull;
    sh.bcolmax[i] = 0ull;
  }
  __syncthreads();
  // Blocks of A_kk and B_ll; consecutive 1x1 blocks are merged in pairs (merge_blocks,
  // merge_blocks_long at tile capacity 64).  Without a B term the columns are
  // independent and stay 1x1.
  constexpr bool kMerge = SYLV_MERGE_DIAG;
  if (warp == 0) {
    int pb = scan_blocks<T, LDY>(Ak, mt, sh.rowblk, sh.astart, lane);
    if (kMerge) {
      __syncwarp();
      pb = TT <= 32 ? merge_blocks(sh.rowblk, sh.astart, mt, pb, &sh.apsd, lane)
                    : merge_blocks_long(sh.rowblk, sh.astart, mt, pb, &sh.apsd, lane);
    } else if (lane == 0) {
      sh.apsd = 0;
    }
    if (lane == 0) sh.pb = pb;
  } else if (warp == 1) {
    int qb = scan_blocks<T, LDY>(Bk, nt, sh.colblk, sh.bstart, lane);
    if (kMerge && B) {
      __syncwarp();
      qb = TT <= 32 ? merge_blocks(sh.colblk, sh.bstart, nt, qb, &sh.bpsd, lane)
                    : merge_blocks_long(sh.colblk, sh.bstart, nt, qb, &sh.bpsd, lane);
    } else if (lane == 0) {
      sh.bpsd = 0;
    }
    if (lane == 0) sh.qb = qb;
  }
  __syncthreads();
  const int pb = sh.pb, qb = sh.qb;
  if (warp == 0)
    order_blocks(sh.astart, pb, kMerge ? sh.apsd : 0ull, sh.aord, sh.acnt, lane);
  else if (warp == 1)
    order_blocks(sh.bstart, qb, kMerge ? sh.bpsd : 0ull, sh.bord, sh.bcnt, lane);
  if (tid == 0) {
    int acc = 0;
    for (int lb = 0; lb < qb; ++lb) {
      sh.qb2[lb] = acc;
      const int nb = sh.bstart[lb + 1] - sh.bstart[lb];
      acc += nb * nb;
    }
    sh.qb2[qb] = acc;
    int off = 0;
    for (int kb = 0; kb < pb; ++kb) {
      sh.pa[kb] = off;
      const int ma = sh.astart[kb + 1] - sh.astart[kb];
      off += ma * ma * acc + ma * nt;
    }
    sh.pa[pb] = off;
  }
  if (ROBUST) {
    // acolmax: rows above each A block; bcolmax: columns right of each B block.
    for (int idx = tid; idx < pb * TT; idx += kThreads) {
      const int kb = idx / TT, r = idx % TT;
      const int ra = sh.astart[kb], re = sh.astart[kb + 1];
      if (r < ra) {
        T sum = T(0);  // binary32 tiles: summed rounded upwards, an upper bound
        for (int i = ra; i < re; ++i) sum = add_up(sum, fabs(Ak[r + i * LDY]));
        atomicMax(&sh.acolmax[kb], abs_bits(static_cast<double>(sum)));
      }
    }
    for (int idx = tid; idx < qb * TT; idx += kThreads) {
      const int lb = idx / TT, c = idx % TT;
      const int j0 = sh.bstart[lb], j1 = sh.bstart[lb + 1];
      if (c >= j1 && c < nt) {
        T sum = T(0);
        for (int j = j0; j < j1; ++j) sum = add_up(sum, fabs(Bk[j + c * LDY]));
        atomicMax(&sh.bcolmax[lb], abs_bits(static_cast<double>(sum)));
      }
    }
  }
  __syncthreads();
  // Pairs enumerated kind by kind (A kind major, then B kind; order_blocks).
  const int na0 = sh.acnt[0], na1 = sh.acnt[1], nb0 = sh.bcnt[0], nb1 = sh.bcnt[1];
  for (int pidx = tid; pidx < pb * qb; pidx += kThreads) {
    int r = pidx, ao = 0, na = na0;
    if (r >= na0 * qb) {
      r -= na0 * qb;
      ao = na0;
      na = na1;
      if (r >= na1 * qb) {
        r -= na1 * qb;
        ao = na0 + na1;
        na = pb - na0 - na1;
      }
    }
    // within this A kind: B kinds in turn, each a na x (blocks of that kind) class
    int bo = 0, nbk = nb0;
    if (r >= na * nb0) {
      r -= na * nb0;
      bo = nb0;
      nbk = nb1;
      if (r >= na * nb1) {
        r -= na * nb1;
        bo = nb0 + nb1;
        nbk = qb - nb0 - nb1;
      }
    }
    const int kb = sh.aord[ao + r / nbk], lb = sh.bord[bo + r % nbk];
    const int ra = sh.astart[kb], ma = sh.astart[kb + 1] - ra;
    const int cb0 = sh.bstart[lb], nb = sh.bstart[lb + 1] - cb0;
    // the blocks' entries in the store's precision (no binary64 instruction in the
    // binary32 kernel, where each would cost 64 binary32 ones)
    FactT a[4], b[4];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        a[i + 2 * j] = (i < ma && j < ma) ? static_cast<FactT>(Ak[(ra + i) + (ra + j) * LDY]) : FactT(0);
        b[i + 2 * j] = (i < nb && j < nb) ? static_cast<FactT>(Bk[(cb0 + i) + (cb0 + j) * LDY]) : FactT(0);
      }
    const bool psa = kMerge && ((sh.apsd >> kb) & 1ull), psb = kMerge && ((sh.bpsd >> lb) & 1ull);
    FactT* fo = fact + pair_offset(sh, kb, lb, ma);
    // Computed in the store's precision (binary32 for the binary32 kernel: an inverse
    // whose norm overflows it is infinite, which sends the pair to the guarded path).
    int pack;
    if (psa && psb)
      pack = pair_quad_prepare<FactT>(a, b, smin, fo);
    else if (psa || psb)
      pack = pair_half_prepare<FactT>(ma, nb, psa, a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3], smin, fo);
    else if (ma == 1 && nb == 1)
      pack = pair_prepare<1, 1, FactT>(a, b, smin, fo);
    else if (ma == 2 && nb == 1)
      pack = pair_prepare<2, 1, FactT>(a, b, smin, fo);
    else if (ma == 1)
      pack = pair_prepare<1, 2, FactT>(a, b, smin, fo);
    else
      pack = pair_prepare<2, 2, FactT>(a, b, smin, fo);
    factp[kb * TT + lb] = pack;
  }
  // Wavefront order of the tile's elements: step s holds the blocks (kb, lb) with
  // (pb-1-kb) + lb = s (without a B term, B null: (pb-1-kb) = s, every column at
  // once), the 2x2-by-2x2 blocks first, then the 2-element ones, then the 1x1 ones,
  // so that a warp's lanes mostly share one dot-product length.
  const int lw = B ? 1 : 0;
  const int nsteps = pb + lw * (qb - 1);
  for (int s = tid; s < nsteps; s += kThreads) {
    int cnt = 0;
    for (int lb = lw ? max(0, s - (pb - 1)) : 0; lb <= (lw ? min(s, qb - 1) : qb - 1); ++lb) {
      const int kb = pb - 1 - (s - lw * lb);
      cnt += (sh.astart[kb + 1] - sh.astart[kb]) * (sh.bstart[lb + 1] - sh.bstart[lb]);
    }
    sh.sstart[s + 1] = static_cast<short>(cnt);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive prefix of the step counts (warp scan, 32 steps a pass)
    int carry = 0;
    if (lane == 0) sh.sstart[0] = 0;
    for (int base = 0; base < nsteps; base += 32) {
      const int st = base + lane;
      int v = st < nsteps ? sh.sstart[st + 1] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (st < nsteps) sh.sstart[st + 1] = static_cast<short>(v + carry);
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  // Every pair writes its own elements: its position within its step counts the
  // step's pairs that come first (more elements, or as many and further left).
  for (int pidx = tid; pidx < pb * qb; pidx += kThreads) {
    const int kb = pidx / qb, lb = pidx % qb;
    const int ra = sh.astart[kb], ma = sh.astart[kb + 1] - ra;
    const int cb0 = sh.bstart[lb], nb = sh.bstart[lb + 1] - cb0;
    const int sz = ma * nb;
    const int s = (pb - 1 - kb) + lw * lb;
    int pos = sh.sstart[s];
    const int lo = lw ? max(0, s - (pb - 1)) : 0, hi = lw ? min(s, qb - 1) : qb - 1;
    for (int l2 = lo; l2 <= hi; ++l2) {
      const int k2 = pb - 1 - (s - lw * l2);
      const int sz2 = (sh.astart[k2 + 1] - sh.astart[k2]) * (sh.bstart[l2 + 1] - sh.bstart[l2]);
      if (sz2 > sz || (sz2 == sz && l2 < lb)) pos += sz2;
    }
    for (int jc = 0; jc < nb; ++jc)
      for (int ir = 0; ir < ma; ++ir)
        sh.eord[pos + ir + ma * jc] = static_cast<unsigned short>((ra + ir) | ((cb0 + jc) << 6) | ((ir + ma * jc) << 12));
  }
  __syncthreads();
}

// Diagonal-tile solve: Algorithm 2 applied to one tile, in wavefront order over its
// 1x1/2x2 blocks.  The blocks (kb, lb) on the anti-diagonal s = (pb-1-kb) + lb are
// independent (without a B term, step s is block row pb-1-s in every column).
//
// Left-looking phase.  Step s forms each of its elements' complete right-hand side
//   r = Y0 - A(row, rows below its block) Z(those rows, col) - Z(row, cols left of its
//       block) B(those cols, col)
// from elements solved in earlier steps: a dot product split across L lanes and summed
// by shuffles, so the FP64 work is dense (a fixed per-element ownership would issue a
// warp instruction whenever any of its lanes has a term).  The block's stored inverse
// then gives its solution (the members of a block sit in one warp and exchange their
// right-hand sides by shuffles).  Robustness: every partial sum is bounded by
//   U0 + (RA + CB) max|Z|,  RA = sum_kb acolmax[kb],  CB = sum_lb bcolmax[lb]
// (U0 bounds |Y0|; RA bounds the A row sums right of any block, CB the B column sums
// above any block), so while that bound stays two binades under omega' = omega/2 (an
// exponent test after every step) no intermediate can exceed omega' and the step needs
// no scaling, which is the outcome the guards of Algorithm 2 reach as well.  The first
// step where the test fails, or where a block's solution would fail the inverse's
// bound test (the guarded elimination is needed), is taken back: its elements get
// their right-hand sides again, every unsolved element owned below receives the
// contributions of the steps before it, and the right-looking phase continues from
// that step.
//
// Right-looking phase (from the hand-over step; the whole solve when the left-looking
// phase is off).  A step solves its blocks (Phase A: one thread per element, the stored
// inverses; a block whose bound test fails is solved by its first thread with the
// guarded elimination), agrees on one tile-wide power of two (Phase B, only when
// some bound comes near omega), and every unsolved element's owner applies the
// step's contributions (Phase C).  Unsolved elements live in their owners'
// registers; an element is written to shared memory when it becomes the right-hand
// side of the next step, and when it is solved.
// Robustness, element-wise with omega' = omega/2 (so every 1x1/2x2 block's row sum
// stays <= omega): U bounds |y| over unsolved elements (recomputed every step); a
// step's blocks are solved with omega'; the step then scales the whole tile by 2^g
// with g = e_min + zeta such that
//   2^zeta (2^e_min U + As Zm + Zm Bs) <= omega',
// As = max over the step's blocks of the A row sums above them, Bs = max of the B
// column sums right of them, Zm = max |z| of the step's blocks at the common scale.
// When all exponents are far from omega' the decision is taken from the exponent
// fields alone (g = e_min = 0, no FP64 work); otherwise warp 0 evaluates
// ProtectUpdate.
template <int TT, typename T, bool ROBUST>
__device__ void diag_solve(DagSmem<TT, T>& sh, int mt, int nt, double omega, double smin, const double* gfact,
                           const int* gfactp, bool nob) {
  constexpr int LDY = DagSmem<TT, T>::LDY;
  constexpr int CSTEP = kThreads / TT;
  constexpr int NC = TT / CSTEP;  // columns owned per thread
  constexpr int NW = kThreads / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  using FactT = typename DagSmem<TT, T>::FactT;
  const FactT* fact;
  const int* factp;
  if constexpr (DagSmem<TT, T>::kFactSmem) {
    fact = sh.fact;
    factp = sh.factp;
  } else {
    fact = gfact;
    factp = gfactp;
  }
  const T* Ak = sh.L;
  const T* Bk = sh.R;
  T* Ys = sh.Y;
  const int pb = sh.pb, qb = sh.qb;
  const double omh = 0.5 * omega;
  const int eo = floor_log2(omh);
  // Without a B term (nob) the columns are independent: step s solves block row
  // pb-1-s in every column block, and no element takes a B-side contribution.
  const int lw = nob ? 0 : 1;

  // Element ownership of the right-looking phase: row tid % TT, columns
  // tid / TT + j * CSTEP (j < NC).
  const int my_r = tid % TT;
  const int my_c0 = tid / TT;
  const bool row_ok = my_r < mt;
  const int kb_r = row_ok ? sh.rowblk[my_r] : 0;
  const int dr = pb - 1 - kb_r;  // distance of this row's block from the bottom
  bool okj[NC];
  int lbcj[NC];
  T yv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int c = my_c0 + j * CSTEP;
    okj[j] = row_ok && c < nt;
    lbcj[j] = okj[j] ? sh.colblk[c] : 0;
  }

  // Initial U (and a pre-scaling if the tile exceeds omega').
  if (ROBUST) {
    unsigned um = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j)
      if (okj[j]) um = max(um, hi_bound(Ys[my_r + (my_c0 + j * CSTEP) * LDY]));
    um = __reduce_max_sync(0xffffffffu, um);
    if (lane == 0) sh.wmax[warp] = um;
  }
  if (tid == 0) {
    sh.e_diag = 0;
    sh.slow = 0;
  }
  __syncthreads();
  if (ROBUST) {
    unsigned u0 = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) u0 = max(u0, sh.wmax[w]);
    const double U0 = from_hi_bound(u0);
    if (U0 > omh) {  // keep every element within omega'
      const int z = floor_log2(omh) - ceil_log2(U0);
      unsigned um = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (okj[j]) {
          T* yp = &Ys[my_r + (my_c0 + j * CSTEP) * LDY];
          *yp = mul2(*yp, z);
          um = max(um, hi_bound(*yp));
        }
      if (tid == 0) sh.e_diag = z;
      um = __reduce_max_sync(0xffffffffu, um);
      __syncthreads();
      if (lane == 0) sh.wmax[warp] = um;
      __syncthreads();
    }
  }
  bool near = false;
  int local_scale_events = 0;
  const int nsteps = pb + lw * (qb - 1);
  int s0 = 0;  // first step of the right-looking phase

  if constexpr (SYLV_LEFT_DIAG) {
    // Exponent bounds of the left-looking test: U0, and RA, CB (a sum of at most TT
    // terms, each below 2^max, is below 2^(max + log2 TT)).
    constexpr int kSumE = (TT <= 32) ? 5 : 6;
    int U0e = 0, RCe = 0;
    if (ROBUST) {
      unsigned u0 = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) u0 = max(u0, sh.wmax[w]);
      U0e = ub_log2(from_hi_bound(u0));
      int ra = -1100;
      for (int b = lane; b < pb; b += 32) ra = max(ra, ub_log2(bits_to_double(sh.acolmax[b])));
      for (int b = lane; b < qb && lw; b += 32) ra = max(ra, ub_log2(bits_to_double(sh.bcolmax[b])));
      RCe = __reduce_max_sync(0xffffffffu, ra) + kSumE + 1;  // RA + CB <= 2 max(RA, CB)
    }
    int zrun = -1100;  // upper bound on log2 max |z| over the solved elements
    s0 = nsteps;
    if (ROBUST && U0e + 2 > eo) s0 = 0;
    // A step's bookkeeping does not depend on the solutions: it is read for step s+1
    // before the barrier that ends step s, so that after the barrier only the dot
    // products, the shuffles and the small solve remain on the step's critical path.
    struct Meta {
      int lg, g, E;          // log2 lanes per element, this thread's element (group), elements of the step
      int r, c, ev, sz;      // element, its index in the block, block size
      int ka0, Ka, Kt;       // first row below the block, A-side terms, all terms
      int fo;                // offset of the block's inverse in the factor store
      FactT fr[4], fn;       // binary32: the element's row of the inverse, and ||Minv||_inf
      bool nr;               // a pivot of the block's small system was raised
    };
    // The binary64 kernels read all of it after the barrier (registers: the prefetch
    // would spill in them, and their steps are bound by the FP64 pipe, not latency).
    constexpr bool kPreF = sizeof(T) == 4;
    constexpr bool kTab = kPreF && DagSmem<TT, T>::kSplitK && TT <= 32;
    unsigned* etab = reinterpret_cast<unsigned*>(sh.kred);
    auto load_inv = [&](Meta& m) {
      const FactT* f = fact + m.fo;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < m.sz) m.fr[u] = f[m.ev * m.sz + u];
      m.fn = f[m.sz * m.sz];
    };
    auto meta = [&](int s, Meta& m) {
      const int e0 = sh.sstart[s];
      m.E = sh.sstart[s + 1] - e0;
      // lanes per element: binary64 aims at about four busy warps (its pipe is the
      // limit), binary32 at all eight (the step's latency is); at most 8, so that the
      // members of a 2x2-by-2x2 block share a warp
      if constexpr (sizeof(T) == 8)
        m.lg = m.E <= 16 ? 3 : m.E <= 32 ? 2 : m.E <= 64 ? 1 : 0;
      else
        m.lg = m.E <= 32 ? 3 : m.E <= 64 ? 2 : m.E <= 128 ? 1 : 0;
      m.g = tid >> m.lg;
      m.r = m.c = m.ev = m.ka0 = m.Ka = m.Kt = m.fo = 0;
      m.sz = 1;
      m.nr = false;
      m.fn = FactT(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) m.fr[u] = FactT(0);
      if (m.g < m.E) {
        const unsigned code = sh.eord[e0 + m.g];
        m.r = code & 63;
        m.c = (code >> 6) & 63;
        m.ev = code >> 12;
        if constexpr (kTab) {
          const unsigned wd = etab[e0 + m.g];
          m.fo = static_cast<int>(wd & 0xffffu);
          m.ka0 = static_cast<int>((wd >> 16) & 63u);
          m.Kt = static_cast<int>((wd >> 22) & 127u);
          m.sz = static_cast<int>((wd >> 29) & 3u) + 1;
          m.nr = (wd >> 31) != 0;
          m.Ka = mt - m.ka0;
        } else {
          const int kb = sh.rowblk[m.r], lb = sh.colblk[m.c];
          const int ra = sh.astart[kb];
          const int ma = sh.astart[kb + 1] - ra;
          const int cb0 = sh.bstart[lb];
          m.sz = ma * (sh.bstart[lb + 1] - cb0);
          m.ka0 = ra + ma;
          m.Ka = mt - m.ka0;
          m.Kt = m.Ka + lw * cb0;
          m.fo = pair_offset(sh, kb, lb, ma);
          m.nr = (factp[kb * TT + lb] & (1 << 16)) != 0;
        }
        if constexpr (kPreF) load_inv(m);
      }
    };
    // The binary32 tile-32 kernel packs each element's bookkeeping into one word per
    // position of the element order, in the split-K buffer (idle during the diagonal
    // solve), so that a step reads it in one round trip instead of a chain of
    // dependent shared-memory loads: the pair's factor-store offset (bits 0-15), the
    // first row below the block (16-21), the number of terms (22-28), the block size
    // minus one (29-30) and whether a pivot was raised (31).
    if constexpr (kTab) {
      if (s0 > 0) {
        const int ne = sh.sstart[nsteps];
        for (int e = tid; e < ne; e += kThreads) {
          const unsigned code = sh.eord[e];
          const int r = code & 63, c = (code >> 6) & 63;
          const int kb = sh.rowblk[r], lb = sh.colblk[c];
          const int ra = sh.astart[kb], ma = sh.astart[kb + 1] - ra;
          const int cb0 = sh.bstart[lb];
          const int sz = ma * (sh.bstart[lb + 1] - cb0);
          const int ka0 = ra + ma;
          const int Kt = (mt - ka0) + lw * cb0;
          const unsigned nr = (static_cast<unsigned>(factp[kb * TT + lb]) >> 16) & 1u;
          etab[e] = static_cast<unsigned>(pair_offset(sh, kb, lb, ma)) | (static_cast<unsigned>(ka0) << 16) |
                    (static_cast<unsigned>(Kt) << 22) | (static_cast<unsigned>(sz - 1) << 29) | (nr << 31);
        }
        __syncthreads();
      }
    }
    Meta m;
    if (kPreF && s0 > 0) meta(0, m);
    for (int s = 0; s < s0; ++s) {
      if constexpr (!kPreF) meta(s, m);
      const int L = 1 << m.lg;
      const int jl = tid & (L - 1);
      const bool act = m.g < m.E;
      // r = Y0 - sum over the element's terms: A side (rows below its block) then B
      // side (columns left of it), one index space split across the group's lanes; the
      // first lane starts from Y0.  Both sides read the left factor with stride LDY and
      // the right one with stride 1.
      T acc = T(0);
      if (act) {
        if (jl == 0) acc = Ys[m.r + m.c * LDY];
        const T* xa = Ak + m.r + m.ka0 * LDY;
        const T* ya = Ys + m.ka0 + m.c * LDY;
        const T* xb = Ys + m.r - m.Ka * LDY;
        const T* yb = Bk + m.c * LDY - m.Ka;
        for (int t = jl; t < m.Kt; t += L) {
          const bool sa = t < m.Ka;
          acc = fma(-(sa ? xa : xb)[t * LDY], (sa ? ya : yb)[t], acc);
        }
      }
      for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const T rhs = acc;
      // the block's right-hand sides, from its members' first lanes
      const int gl = ((m.g - m.ev) << m.lg) & 31;
      T rt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) rt[u] = __shfl_sync(0xffffffffu, rhs, u < m.sz ? gl + (u << m.lg) : lane);
      bool bad = false;
      unsigned hb = 0;
      const int r = m.r, c = m.c;
      if (act) {
        if constexpr (!kPreF) load_inv(m);
        if (m.nr) near = true;
        int rexp = -1022;
        FactT z = FactT(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < m.sz) {
            rexp = max(rexp, ub_log2(rt[u]));
            z = fma(m.fr[u], static_cast<FactT>(rt[u]), z);
          }
        bad = ROBUST && ub_log2(m.fn) + rexp + 1 > eo;
        const T zt = static_cast<T>(z);
        if (!bad) {
          if (jl == 0) Ys[r + c * LDY] = zt;
          hb = hi_bound(zt);
        }
      }
      if (ROBUST) {
        hb = __reduce_max_sync(0xffffffffu, hb);
        if (lane == 0) sh.wz[s & 1][warp] = hb;
      }
      if (kPreF && s + 1 < s0) meta(s + 1, m);
      const int anybad = __syncthreads_or(bad);
      if (ROBUST) {
        unsigned zb = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) zb = max(zb, sh.wz[s & 1][w]);
        zrun = max(zrun, ub_log2(from_hi_bound(zb)));
        if (anybad || max(U0e, RCe + zrun) + 2 > eo) {
          // hand this step to the right-looking phase: its elements get their
          // right-hand sides back
          if (act && jl == 0) Ys[r + c * LDY] = rhs;
          s0 = s;
          __syncthreads();
        }
      }
    }
  }

  if constexpr (ROBUST || !SYLV_LEFT_DIAG) {
    if (s0 < nsteps) {
      // Owned unsolved elements into registers, with the contributions of the steps
      // before s0 (solved in the left-looking phase): the X bottom blocks of their
      // column and the Yb left blocks of their row.  The bound test of step s0 - 1
      // covers these sums.
      unsigned um = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        yv[j] = T(0);
        if (!okj[j]) continue;
        const int c = my_c0 + j * CSTEP;
        const int dd = dr + lw * lbcj[j];
        if (dd < s0) continue;
        T y = Ys[my_r + c * LDY];
        if (dd > s0 && s0 > 0) {
          const int X = s0 - lw * lbcj[j];
          if (X > 0)
            for (int t = sh.astart[pb - X]; t < mt; ++t) y = fma(-Ak[my_r + t * LDY], Ys[t + c * LDY], y);
          const int Yb = s0 - dr;
          if (lw && Yb > 0)
            for (int t = 0; t < sh.bstart[Yb]; ++t) y = fma(-Ys[my_r + t * LDY], Bk[t + c * LDY], y);
        }
        yv[j] = y;
        if (ROBUST) um = max(um, hi_bound(y));
      }
      if (ROBUST) {
        um = __reduce_max_sync(0xffffffffu, um);
        if (lane == 0) sh.wmax[warp] = um;
      }
      __syncthreads();
    }
  for (int s = s0; s < nsteps; ++s) {
    // Phase C's coefficients do not depend on this step's solutions: the binary32
    // tile-32 kernel (latency bound, with registers to spare) fetches them now, while
    // Phase A runs; the others read them after the barrier.  The block solved in
    // column block lbc lies at block row pb-1-(s-lbc); the one solved in this row's
    // block row at column block s-dr.
    constexpr bool kPre = sizeof(T) == 4 && TT <= 32;
    constexpr int NP = kPre ? NC : 1;
    const int lbs = s - dr;
    const bool bs_ok = lw && row_ok && lbs >= 0 && lbs < qb;
    int cs0 = 0, nbs = 0;
    if (bs_ok) {
      cs0 = sh.bstart[lbs];
      nbs = sh.bstart[lbs + 1] - cs0;
    }
    T ca0[NP], ca1[NP], cb0[NP], cb1[NP];
    int rsj[NP];
    unsigned amask = 0, a2mask = 0, bmask = 0;  // per slot: A side present / 2 rows; B side present
    // The warps holding this step's Phase A threads fetch after the barrier instead:
    // their Phase A is the step's critical path.
    const int e0 = sh.sstart[s];
    const int nact = sh.sstart[s + 1] - e0;
    const bool pre_early = warp >= ((nact + 31) >> 5);
    auto prefetch = [&]() {
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int c = my_c0 + j * CSTEP;
        const int lbc = lbcj[j];
        const int ia = s - lw * lbc;
        ca0[j] = ca1[j] = cb0[j] = cb1[j] = T(0);
        rsj[j] = 0;
        if (okj[j] && dr + lw * lbc > s) {
          if (ia >= 0 && ia < dr) {
            const int kbs = pb - 1 - ia;
            const int rs0 = sh.astart[kbs];
            rsj[j] = rs0;
            amask |= 1u << j;
            ca0[j] = Ak[my_r + rs0 * LDY];
            if (sh.astart[kbs + 1] - rs0 == 2) {
              a2mask |= 1u << j;
              ca1[j] = Ak[my_r + (rs0 + 1) * LDY];
            }
          }
          if (bs_ok && lbs < lbc) {
            bmask |= 1u << j;
            cb0[j] = Bk[cs0 + c * LDY];
            if (nbs == 2) cb1[j] = Bk[cs0 + 1 + c * LDY];
          }
        }
      }
    };
    if constexpr (kPre)
      if (pre_early) prefetch();
    // Phase A: the step's elements, one thread each.  All reads of the step's
    // right-hand sides come before any write of a solution (__syncwarp).
    const bool act = tid < nact;
    int r = 0, c = 0, e = 0, r0 = 0, c0 = 0, ma = 1, sz = 0, lb = 0, eb = 0, mode = 0;
    double rv[4] = {0.0, 0.0, 0.0, 0.0};
    FactT z = FactT(0);
    if (act) {
      const unsigned code = sh.eord[e0 + tid];
      r = code & 63;
      c = (code >> 6) & 63;
      e = code >> 12;
      const int kb = sh.rowblk[r];
      lb = sh.colblk[c];
      r0 = sh.astart[kb];
      ma = sh.astart[kb + 1] - r0;
      c0 = sh.bstart[lb];
      const int nb = sh.bstart[lb + 1] - c0;
      sz = ma * nb;
      const FactT* f = fact + pair_offset(sh, kb, lb, ma);
      if (factp[kb * TT + lb] & (1 << 16)) near = true;
      T rt[4];
      int rexp = -1022;  // upper bound on log2 max |r| (exponent fields only)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        rt[u] = (u < sz) ? Ys[(r0 + (ma == 2 ? (u & 1) : 0)) + (c0 + (ma == 2 ? (u >> 1) : u)) * LDY] : T(0);
        rexp = max(rexp, ub_log2(rt[u]));
      }
      const bool ok = !ROBUST || ub_log2(f[sz * sz]) + rexp + 1 <= eo;
      if (ok) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < sz) z = fma(f[e * sz + u], static_cast<FactT>(rt[u]), z);
        mode = 1;
        if (ROBUST) {
          unsigned u0 = 0;
#pragma unroll
          for (int w = 0; w < NW; ++w) u0 = max(u0, sh.wmax[w]);
          const int ez = ub_log2(z);
          const bool fast = ub_log2(from_hi_bound(u0)) + 2 <= eo &&
                            ub_log2(bits_to_double(sh.acolmax[kb])) + ez + 2 <= eo &&
                            ez + ub_log2(bits_to_double(sh.bcolmax[lb])) + 2 <= eo;
          if (!fast) sh.slow = 1;
        }
      } else if (e == 0) {
        // Guarded small solve of the whole block by its first thread (rare).  A pseudo
        // block takes the same guarded elimination of its (block-triangular) system.
#pragma unroll
        for (int u = 0; u < 4; ++u) rv[u] = to_f64(rt[u]);
        double a[4], b[4];
        for (int i = 0; i < 2; ++i)
          for (int jj = 0; jj < 2; ++jj) {
            a[i + 2 * jj] = (i < ma && jj < ma) ? static_cast<double>(Ak[(r0 + i) + (r0 + jj) * LDY]) : 0.0;
            b[i + 2 * jj] = (i < nb && jj < nb) ? static_cast<double>(Bk[(c0 + i) + (c0 + jj) * LDY]) : 0.0;
          }
        double lu[20];
        const bool psa = SYLV_MERGE_DIAG && ((sh.apsd >> kb) & 1ull);
        const bool psb = SYLV_MERGE_DIAG && ((sh.bpsd >> lb) & 1ull);
        const int pack = pair_factor(ma, nb, psa, psb, a, b, smin, lu);
        double rg[4] = {rv[0], rv[1], rv[2], rv[3]};  // the guarded solve takes its own copy
        if (sz == 1)
          eb = pair_solve_guarded<1>(lu, pack, rg, omh, eo, true);
        else if (sz == 2)
          eb = pair_solve_guarded<2>(lu, pack, rg, omh, eo, true);
        else
          eb = pair_solve_guarded<4>(lu, pack, rg, omh, eo, true);
#pragma unroll
        for (int u = 0; u < 4; ++u) rv[u] = rg[u];
        mode = 2;
        sh.slow = 1;
      }
    }
    __syncwarp();
    if (mode == 1) {
      Ys[r + c * LDY] = static_cast<T>(z);
    } else if (mode == 2) {
#pragma unroll
      for (int u = 0; u < 4; ++u)  // static indices keep rv in registers
        if (u < sz) Ys[(r0 + (ma == 2 ? (u & 1) : 0)) + (c0 + (ma == 2 ? (u >> 1) : u)) * LDY] = static_cast<T>(rv[u]);
    }
    if (mode != 0 && e == 0) {
      sh.pe[lb] = eb;
      sh.pr0[lb] = static_cast<short>(r0);
      sh.pma[lb] = static_cast<short>(ma);
    }
    __syncthreads();
    if constexpr (kPre)
      if (!pre_early) prefetch();
    const int lb_lo = lw ? max(0, s - (pb - 1)) : 0;
    const int lb_hi = lw ? min(s, qb - 1) : qb - 1;
    int g = 0;
    if (ROBUST && sh.slow) {
      // Phase B (rare): exact tile-wide factor of this step.
      if (warp == 0) {
        int emin = 0;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) emin = min(emin, sh.pe[lb]);
        emin = warp_min(emin);
        double zs = 0.0, as = 0.0, bs = 0.0;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) {
          const int kb = pb - 1 - (s - lw * lb);
          const int r0 = sh.astart[kb], ma = sh.astart[kb + 1] - r0;
          const int c0 = sh.bstart[lb], nb = sh.bstart[lb + 1] - c0;
          double zm = 0.0;
          for (int jj = 0; jj < nb; ++jj)
            for (int i = 0; i < ma; ++i) zm = fmax(zm, fabs(static_cast<double>(Ys[(r0 + i) + (c0 + jj) * LDY])));
          zs = fmax(zs, mul2(zm, emin - sh.pe[lb]));
          as = fmax(as, bits_to_double(sh.acolmax[kb]));
          bs = fmax(bs, bits_to_double(sh.bcolmax[lb]));
        }
        zs = warp_max(zs);
        as = warp_max(as);
        bs = warp_max(bs);
        if (lane == 0) {
          unsigned u0 = 0;
          for (int w = 0; w < NW; ++w) u0 = max(u0, sh.wmax[w]);
          const double U1 = mul2(from_hi_bound(u0), emin);
          const int z1 = protect_update(U1, as, zs, omh);
          const double zs1 = mul2(zs, z1);
          const double U2 = mul2(U1, z1) + as * zs1;
          const int z2 = protect_update(U2, zs1, bs, omh);
          const int gg = emin + z1 + z2;
          sh.e_diag += gg;
          sh.g = gg;
          if (gg != 0) ++local_scale_events;
        }
        __syncwarp();
        const int gg = sh.g;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) {
          const int sc = gg - sh.pe[lb];
          if (sc != 0) {
            const int kb = pb - 1 - (s - lw * lb);
            const int r0 = sh.astart[kb], ma = sh.astart[kb + 1] - r0;
            const int c0 = sh.bstart[lb], nb = sh.bstart[lb + 1] - c0;
            for (int jj = 0; jj < nb; ++jj)
              for (int i = 0; i < ma; ++i) {
                T* yp = &Ys[(r0 + i) + (c0 + jj) * LDY];
                *yp = mul2(*yp, sc);
              }
          }
        }
      }
      __syncthreads();
      g = sh.g;
      // Every thread has read the flag before the barrier above; clearing it earlier
      // (in warp 0) would let a later warp skip this phase and its barrier.
      if (tid == 0) sh.slow = 0;
    }
    // Phase C: every owned unsolved element takes the scale and this step's
    // contributions: the block solved in its column block below it (A side) and the
    // block solved in its row block left of it (B side).
    T zb0 = T(0), zb1 = T(0);
    if (bs_ok) {
      zb0 = Ys[my_r + cs0 * LDY];
      if (nbs == 2) zb1 = Ys[my_r + (cs0 + 1) * LDY];
    }
    unsigned wm = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = my_c0 + j * CSTEP;
      const int lbc = lbcj[j];
      const int dd = dr + lw * lbc;
      if (!okj[j]) continue;
      if (dd < s) {
        if (g != 0) {  // solved earlier: rescale in place (rare)
          T* yp = &Ys[my_r + c * LDY];
          *yp = mul2(*yp, g);
        }
      } else if (dd > s) {
        T y = yv[j];
        if (g != 0) y = mul2(y, g);
        if constexpr (kPre) {
          if (amask & (1u << j)) {  // block of column block lbc solved now, below this row
            y = fma(-ca0[j], Ys[rsj[j] + c * LDY], y);
            if (a2mask & (1u << j)) y = fma(-ca1[j], Ys[rsj[j] + 1 + c * LDY], y);
          }
          if (bmask & (1u << j)) {  // block of this row block solved now, left of this column
            y = fma(-zb0, cb0[j], y);
            if (nbs == 2) y = fma(-zb1, cb1[j], y);
          }
        } else {
          const int ia = s - lw * lbc;
          if (ia >= 0 && ia < dr) {  // block of column block lbc solved now, below this row
            const int rs0 = sh.pr0[lbc];
            y = fma(-Ak[my_r + rs0 * LDY], Ys[rs0 + c * LDY], y);
            if (sh.pma[lbc] == 2) y = fma(-Ak[my_r + (rs0 + 1) * LDY], Ys[rs0 + 1 + c * LDY], y);
          }
          if (bs_ok && lbs < lbc) {  // block of this row block solved now, left of this column
            y = fma(-zb0, Bk[cs0 + c * LDY], y);
            if (nbs == 2) y = fma(-zb1, Bk[cs0 + 1 + c * LDY], y);
          }
        }
        yv[j] = y;
        if (dd == s + 1) Ys[my_r + c * LDY] = y;  // right-hand side of the next step
        if (ROBUST) wm = max(wm, hi_bound(y));
      }
    }
    if (ROBUST) {
      wm = __reduce_max_sync(0xffffffffu, wm);
      if (lane == 0) sh.wmax[warp] = wm;
    }
    __syncthreads();
  }
  }
  if (near) atomicOr(&sh.flags, kFlagNearSingular);
  if (local_scale_events) atomicAdd(&sh.nscale, local_scale_events);
}

// ----------------------------------------------------------------------------
// GEMM operand staging: L (rows x kdim) from column-major P (coalesced along rows),
// R (kdim x cols) from column-major P (coalesced along k); both stored k-major at
// the given k offset.  Only rows kk < kdim are written (groups stage back to back).
template <int TT, typename T, bool FROM_Y>
__device__ __forceinline__ void stage_left(T* L, const T* P, int64_t ld, int rows, int kdim) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
  for (int idx = threadIdx.x; idx < TT * kdim; idx += kThreads) {
    const int r = idx % TT, kk = idx / TT;
    T v = T(0);
    if (r < rows) {
      const T* src = P + r + kk * ld;
      v = FROM_Y ? __ldcg(src) : __ldg(src);
    }
    L[kk * LDG + r] = v;
  }
}
template <int TT, typename T, bool FROM_Y>
__device__ __forceinline__ void stage_right(T* R, const T* P, int64_t ld, int kdim, int cols) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
  for (int idx = threadIdx.x; idx < TT * kdim; idx += kThreads) {
    const int kk = idx % kdim, c = idx / kdim;
    T v = T(0);
    if (c < cols) {
      const T* src = P + kk + c * ld;
      v = FROM_Y ? __ldcg(src) : __ldg(src);
    }
    R[kk * LDG + c] = v;
  }
}

// acc -= L * R over kk < kdim; thread (tx, ty) owns rows tx*MR.., columns ty*NR..
// Operands are read two elements at a time (rbase, cbase and LDG are even, so each
// pair is 8-byte aligned in binary32 and 16-byte aligned in binary64): half the
// shared-memory load instructions of scalar reads, which bound this loop.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};
template <int TT, typename T, int MR, int NR>
__device__ __forceinline__ void gemm_sub(T (&acc)[MR][NR], const T* L, const T* R, int kdim, int rbase,
                                         int cbase) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
  static_assert(MR % 2 == 0 && NR % 2 == 0 && LDG % 2 == 0, "paired operand reads");
  using V2 = typename Vec2<T>::type;
#pragma unroll 4
  for (int kk = 0; kk < kdim; ++kk) {
    T a[MR], b[NR];
#pragma unroll
    for (int i = 0; i < MR; i += 2) {
      const V2 v = *reinterpret_cast<const V2*>(&L[kk * LDG + rbase + i]);
      a[i] = v.x;
      a[i + 1] = v.y;
    }
#pragma unroll
    for (int j = 0; j < NR; j += 2) {
      const V2 v = *reinterpret_cast<const V2*>(&R[kk * LDG + cbase + j]);
      b[j] = v.x;
      b[j + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
  }
}

// The binary32 tile-32 group product.  With one 2x2 block per thread (gemm_sub) a
// warp needs two shared-memory wavefronts per four FFMA instructions, which caps the
// FP32 pipe at half its rate.  Here four groups of 64 threads each take every fourth
// k with a 4x4 block per thread (four wavefronts per sixteen FFMA), write their
// partial tiles to kred, and every thread sums the four partials of its own 2x2
// block in group order (deterministic).  part receives -sum_k L[k, r] R[k, c], as
// gemm_sub does; the caller's barrier after the accumulation frees kred again.
template <int TT, typename T>
__device__ __forceinline__ void gemm_sub_split4(T (&part)[2][2], const T* L, const T* R, int kdim, int rbase,
                                                int cbase, T* kred) {
  static_assert(sizeof(T) == 4 && TT == 32 && kThreads == 256, "binary32, tile 32, 256 threads");
  constexpr int LDG = DagSmem<TT, T>::LDG;
  static_assert(LDG % 2 == 0, "paired operand reads");
  const int tid = threadIdx.x;
  const int g = tid >> 6, t = tid & 63;
  const int r4 = (t & 7) * 4, c4 = (t >> 3) * 4;
  T p[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) p[i][j] = T(0);
#pragma unroll 2
  for (int kk = g; kk < kdim; kk += 4) {
    const float2 a01 = *reinterpret_cast<const float2*>(&L[kk * LDG + r4]);
    const float2 a23 = *reinterpret_cast<const float2*>(&L[kk * LDG + r4 + 2]);
    const float2 b01 = *reinterpret_cast<const float2*>(&R[kk * LDG + c4]);
    const float2 b23 = *reinterpret_cast<const float2*>(&R[kk * LDG + c4 + 2]);
    const T a[4] = {a01.x, a01.y, a23.x, a23.y};
    const T b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) p[i][j] = fma(-a[i], b[j], p[i][j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    *reinterpret_cast<float4*>(&kred[g * TT * TT + (c4 + j) * TT + r4]) = make_float4(p[0][j], p[1][j], p[2][j], p[3][j]);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float2 s = *reinterpret_cast<const float2*>(&kred[(cbase + j) * TT + rbase]);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      const float2 v = *reinterpret_cast<const float2*>(&kred[q * TT * TT + (cbase + j) * TT + rbase]);
      s.x += v.x;
      s.y += v.y;
    }
    part[0][j] = s.x;
    part[1][j] = s.y;
  }
}

// Infinity norm of the tile in sh.Y (mt x nt) into sh.umax (bit pattern, atomic
// maximum; sh.umax zeroed before).  A warp per row, lanes across the columns and a
// shuffle tree, so the sum is a short dependency chain; the maximum is taken on the
// bit patterns of the non-negative sums, so a NaN row still shows.  Binary32 tiles
// sum in binary32 rounded upwards (an upper bound), without binary64 instructions.
template <int TT, typename T>
__device__ __forceinline__ void tile_norm_max(DagSmem<TT, T>& sh, int mt, int nt) {
  constexpr int LDY = DagSmem<TT, T>::LDY;
  const int wq = threadIdx.x >> 5, lq = threadIdx.x & 31;
  T mx = T(0);
  for (int r = wq; r < mt; r += kThreads / 32) {
    T s = T(0);
    for (int c = lq; c < nt; c += 32) s = add_up(s, fabs(sh.Y[r + c * LDY]));
    for (int o = 16; o > 0; o >>= 1) s = add_up(s, __shfl_xor_sync(0xffffffffu, s, o));
    mx = mag_bits(s) > mag_bits(mx) ? s : mx;
  }
  if (lq == 0 && mag_bits(mx)) atomicMax(&sh.umax, abs_bits(static_cast<double>(mx)));
}

template <int TT, typename T, bool ROBUST>
__global__ void __launch_bounds__(kThreads, 2) dag_kernel(Work w) {
  static_assert(TT == 32 || TT == 64, "tile capacity");
  constexpr int MR = TT / 16, NR = TT / 16;
  constexpr int LDY = DagSmem<TT, T>::LDY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DagSmem<TT, T>& sh = *reinterpret_cast<DagSmem<TT, T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int rbase = tx * MR, cbase = ty * NR;
  Ctrl* ctrl = w.ctrl;
  if (w.skip && ld_volatile(w.skip)) return;
  // SM cap: the CTAs placed on SMs outside the budget leave before their first ticket
  // (tickets are dynamic, so the others take all the tasks).  CTAs inside the budget
  // register; CTA 0, if outside, leaves once one has registered and works itself if
  // none has within 2 ms, so the kernel is never left without a worker.  The whole
  // CTA shares one SM id, so every exit is CTA-uniform.
  if (w.sm_limit > 0) {
    const bool inside = static_cast<int>(sm_id()) < w.sm_limit;
    if (inside) {
      if (tid == 0) atomicAdd(&ctrl->workers, 1);
    } else if (blockIdx.x != 0) {
      return;
    } else {
      if (tid == 0) {
        const unsigned long long t0 = global_ns();
        int seen = 0;
        while (!(seen = ld_volatile(&ctrl->workers)) && global_ns() - t0 < 2000000ull) __nanosleep(1000);
        sh.abort = seen;
      }
      __syncthreads();
      if (sh.abort) return;
    }
  }
  const bool packed = w.pack != nullptr;
  uint32_t stage_phase = 0;
  if (packed) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sh.stage_bar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }

  for (;;) {
    if (tid == 0) {
      const int tk = atomicAdd(&ctrl->ticket, 1);
      sh.task = (tk < ctrl->ntasks && ld_volatile(&ctrl->err) == 0) ? tk : -1;
      sh.abort = 0;
      sh.flags = 0;
      sh.nscale = 0;
      sh.skipt = 0;
      if (sh.task >= 0 && w.eqskip) {
        // A converged equation of a batched refinement: its tiles are only marked
        // final (every consumer belongs to the same equation and skips as well).
        const Task t0 = w.tasks[sh.task];
        if (ld_volatile(w.eqskip + static_cast<int64_t>(t0.inst) * w.eqskip_stride)) {
          st_release64(w.tflag + w.inst[t0.inst].tile + t0.tile, tile_word(0, 0.0));
          sh.skipt = 1;
        }
      }
    }
    __syncthreads();
    if (sh.task < 0) break;
    if (sh.skipt) {
      __syncthreads();  // thread 0 rewrites sh.task next
      continue;
    }
    const Task task = w.tasks[sh.task];
    const Inst I = w.inst[task.inst];
    InstState* st = &w.st[task.inst];
    const int p = st->p;
    const int k = task.tile / I.qmax, l = task.tile % I.qmax;
    const int32_t* rb = w.ibuf + I.rb;
    const int32_t* cb = w.ibuf + I.cb;
    const int r0 = rb[k], mt = rb[k + 1] - r0;
    const int c0 = cb[l], nt = cb[l + 1] - c0;
    const T* A = static_cast<const T*>(I.A);
    const T* B = static_cast<const T*>(I.B);
    T* C = static_cast<T*>(I.C);
    const double omega = I.omega;
    const double* an = w.dbuf + I.an;
    const double* bn = w.dbuf + I.bn;
    int32_t* texp = w.texp + I.tile;
    unsigned long long* tflag = w.tflag + I.tile;
    double* tnorm = w.tnorm + I.tile;

    double* fact = w.fact + static_cast<int64_t>(blockIdx.x) * w.fact_stride;
    int* factp = w.factp + static_cast<int64_t>(blockIdx.x) * TT * TT;
    diag_prepare<TT, T, ROBUST>(sh, A, I.lda, I.nob ? nullptr : B, I.ldb, r0, c0, mt, nt, st->smin, fact, factp);

    // ---- accumulator <- C_kl, exact infinity norm.  In binary32 the accumulator
    // is compensated: every group's product is summed into a fresh partial and the
    // partials enter (acc, acc_lo) by two-sum, so a tile that receives thousands of
    // products keeps ~binary32 accuracy instead of losing sqrt(K) ulps.
    constexpr bool kComp = std::is_same<T, float>::value;
    T acc[MR][NR];
    T acc_lo[MR][NR];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc_lo[i][j] = T(0);
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const int r = rbase + i, c = cbase + j;
        acc[i][j] = (r < mt && c < nt) ? __ldcg(&C[(r0 + r) + (int64_t)(c0 + c) * I.ldc]) : T(0);
        sh.Y[r + c * LDY] = acc[i][j];
      }
    if (tid == 0) sh.umax = 0ull;
    __syncthreads();
    if (ROBUST) {
      tile_norm_max<TT, T>(sh, mt, nt);
      __syncthreads();
      if (tid == 0) {
        double nb = __longlong_as_double(static_cast<long long>(sh.umax));
        int e0 = 0;
        if (!(nb <= 1.7976931348623157e308)) {
          set_err(st, SYLV_ERR_NONFINITE);
          nb = 0.0;
        } else if (nb > omega) {  // keep C's tile within the precondition of Algorithm 2
          e0 = floor_log2(omega) - ceil_log2(nb);
          nb = mul2(nb, e0);
        }
        sh.e_acc = e0;
        sh.nb_acc = nb;
      }
      __syncthreads();
      if (sh.e_acc != 0) {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[i][j] = mul2(acc[i][j], sh.e_acc);
      }
    } else if (tid == 0) {
      sh.e_acc = 0;
    }

    // ---- incoming updates, producers in anti-diagonal order.  Producer q of the
    // tile (0 <= q < d): while only one side has producers left to start, that side;
    // afterwards A side then B side per anti-diagonal.  Up to G producers whose
    // flags are already set are staged back to back and applied in one GEMM pass;
    // each element still receives their products in producer order.  With equal
    // exponents and bounds far from omega that is the arithmetic of one at a time;
    // otherwise the group takes one exponent and one ProtectUpdate factor (scaling
    // its tiles by exact powers of two), and a lone producer near omega the exact
    // single-producer ProtectUpdate.
    // Without a B term (nob) only the tiles below contribute: d = p-1-k, all on the A side.
    const int lq = I.nob ? 0 : l;
    const int d = (p - 1 - k) + lq;
    const int a0 = lq, b0 = p - 1 - k;
    const int lo = min(a0, b0), hi = max(a0, b0);
    const int eo = floor_log2(omega);
    auto producer = [&](int q, int& side, int& prod, int& kdim) {
      int sd;
      int sq;
      if (q < hi - lo) {
        sd = (a0 < b0) ? 0 : 1;
        sq = lo + q;
      } else {
        const int r = q - (hi - lo);
        sq = hi + r / 2;
        sd = r & 1;
      }
      side = sd;
      if (sd == 0) {
        const int i = p - 1 + lq - sq;  // A side: Y_kl -= A_ki Y_il
        prod = i * I.qmax + l;
        kdim = rb[i + 1] - rb[i];
      } else {
        const int j = sq - (p - 1 - k);  // B side: Y_kl -= Y_kj B_jl
        prod = k * I.qmax + j;
        kdim = cb[j + 1] - cb[j];
      }
    };
    auto opnorm = [&](int side, int prod) {
      return (side == 0) ? an[(int64_t)k * I.pmax + prod / I.qmax] : bn[(int64_t)(prod % I.qmax) * I.qmax + l];
    };
    for (int q = 0; q < d && !sh.abort;) {
      if (tid < 32) {
        // Warp 0 forms the group: lane u looks at producer q + u.  Every candidate's
        // flag (acquire) and operator norm (independent of readiness) are fetched in
        // one round trip; lane 0 then waits for its flag (bounded) if it was not set,
        // and the group is the ready prefix.  Exponents and bounds are read after the
        // acquire that saw their flag set.
        constexpr int G = DagSmem<TT, T>::G;
        const int lane = tid;
        int side = 0, prod = 0, kdim = 0;
        const bool cand = lane < G && q + lane < d;
        if (cand) producer(q + lane, side, prod, kdim);
        unsigned long long fl = cand ? ld_acquire64(&tflag[prod]) : 0ull;
        double on = 0.0;
        if (ROBUST && cand) on = opnorm(side, prod);
        int okw = 1;
        if (lane == 0 && !fl) okw = wait_word(&tflag[prod], ctrl, w.timeout_ns, &fl) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          if (lane == 0) sh.abort = 1;
        } else {
          const bool ready = cand && (lane == 0 || fl != 0);
          const unsigned nr = ~__ballot_sync(0xffffffffu, ready);
          int g = nr ? __ffs(nr) - 1 : 32;  // the ready prefix (lane 0 is ready)
          int fast = 1;
          int ep = 0;
          double pn = 0.0;
          if (ROBUST && lane < g) {  // from the ready word: no second round trip
            ep = word_exp(fl);
            pn = word_norm(fl);
          }
          if (lane >= g) on = 0.0;
          int gsacc = 0;
          if (ROBUST) {
            // The group is applied in one pass (Algorithm 3 on the concatenated update
            // C - [A_1 .. A_g][Y_1; ..; Y_g], bound sum_p ||A_p|| ||Y_p||) at the smallest
            // exponent eta of the accumulator and its producers, times 2^z with z the
            // ProtectUpdate factor of the summed bound.  z = 0 whenever the summed
            // bound of the g + 1 terms at eta stays ceil(log2(g + 1)) binades (at least
            // two) under omega; one-at-a-time Algorithm 3 then reaches the same exponent
            // with no guard firing.  Equal exponents and z = 0 need no scaling;
            // otherwise the accumulator and each producer's Y tile take exact powers of
            // two.  A lone producer that needs a guard takes the exact single-producer
            // ProtectUpdate below.
            const bool same = __all_sync(0xffffffffu, lane >= g || ep == sh.e_acc);
            int emn = lane < g ? ep : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) emn = min(emn, __shfl_xor_sync(0xffffffffu, emn, o));
            const int eta = min(sh.e_acc, emn);
            const int ea = ub_log2(on);
            int emx = lane < g ? ea + ub_log2(pn) + (eta - ep) : -4096;
            for (int o = 16; o > 0; o >>= 1) emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
            emx = max(emx, ub_log2(sh.nb_acc) + (eta - sh.e_acc));
            const int margin = max(2, 32 - __clz(g));
            const bool fits = emx + margin <= eo;
            if (!fits && g == 1) {
              fast = 0;
            } else {
              int z = 0;
              double nb;
              if (fits) {
                const double inc = lane < g ? on * mul2(pn, eta - ep) : 0.0;  // summed in producer order
                nb = mul2(sh.nb_acc, eta - sh.e_acc);
                for (int u = 0; u < g; ++u) nb += __shfl_sync(0xffffffffu, inc, u);
              } else {
                // Terms normalised by 2^-emx (each <= 1, no overflow), multiplied and
                // summed in producer order rounded towards +inf, plus 2^-1000 for any
                // subnormal term, so sn bounds the exact normalised sum from above; z is
                // then the largest power of two with 2^z * sn * 2^emx <= omega.
                const double tn = lane < g ? __dmul_ru(mul2(on, -ea), mul2(pn, (eta - ep) - (emx - ea))) : 0.0;
                double sn = mul2(sh.nb_acc, (eta - sh.e_acc) - emx);
                for (int u = 0; u < g; ++u) sn = __dadd_ru(sn, __shfl_sync(0xffffffffu, tn, u));
                sn = __dadd_ru(sn, 0x1p-1000);
                // omega = 2^eo f, f in [1, 2): z = (eo - emx) + floor(log2(f / sn)), the
                // quotient rounded towards -inf
                z = min(0, (eo - emx) + floor_log2(__ddiv_rd(mul2(omega, -eo), sn)));
                nb = mul2(sn, emx + z);
              }
              fast = (same && z == 0) ? 1 : 2;
              const int delta = eta + z;
              if (lane < g) sh.gsop[lane] = delta - ep;
              gsacc = delta - sh.e_acc;
              const bool scaled = __any_sync(0xffffffffu, (lane < g && ep != delta)) || gsacc != 0;
              __syncwarp();
              if (lane == 0) {
                sh.nb_acc = nb;
                sh.e_acc = delta;
                if (scaled) ++sh.nscale;
              }
            }
          }
          int ko = lane < g ? kdim : 0;  // exclusive prefix of the K extents
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, ko, o);
            if (lane >= o) ko += v;
          }
          // Packed tiles are zero-padded to TT rows of k.  The binary64 kernels stage
          // each producer's own kdim rows back to back (a row of LDG doubles is a
          // multiple of 16 bytes, as bulk copies require), so the group product runs
          // over no padding rows; the binary32 kernels stage whole slots (a binary32 row
          // is not a multiple of 16 bytes).
          constexpr bool kTight = sizeof(T) == 8;
          const bool slots = packed && !kTight;
          const int ktot = slots ? g * TT : __shfl_sync(0xffffffffu, ko, g - 1);
          if (lane < g) {
            sh.gside[lane] = side;
            sh.gprod[lane] = prod;
            sh.gk[lane] = kdim;
            sh.goff[lane] = slots ? lane * TT : ko - kdim;
          }
          if (packed) {
            // The group is staged by bulk copies (async proxy): lane 0 sets the
            // transaction count, then every member's lane issues its own two copies,
            // after its own flag acquire and proxy fences, so the issue runs in
            // parallel instead of 2g copies in a row on one lane.
            constexpr uint32_t kRow = DagSmem<TT, T>::LDG * sizeof(T);
            const uint32_t bytes = kTight ? static_cast<uint32_t>(kdim) * kRow : static_cast<uint32_t>(w.pack_slot);
            const uint32_t total = kTight ? 2u * static_cast<uint32_t>(ktot) * kRow : 2u * g * bytes;
            const uint32_t bar = smem_addr(&sh.stage_bar);
            if (lane == 0)
              asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total)
                           : "memory");
            __syncwarp();
            if (lane < g) {
              asm volatile("fence.proxy.async.global;" ::: "memory");
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the last GEMM's reads
              int64_t sl, sr;
              if (side == 0) {  // A_ki and Y_il
                const int i = prod / I.qmax;
                sl = pack_a(I, k, i);
                sr = pack_yr(I, i, l);
              } else {  // Y_kj and B_jl
                const int j = prod % I.qmax;
                sl = pack_yl(I, k, j);
                sr = pack_b(I, j, l);
              }
              const int dk = slots ? lane * TT : ko - kdim;  // first staged row of this member
              bulk_copy_g2s(sh.L + dk * DagSmem<TT, T>::LDG, w.pack + sl * w.pack_slot, bytes, bar);
              bulk_copy_g2s(sh.R + dk * DagSmem<TT, T>::LDG, w.pack + sr * w.pack_slot, bytes, bar);
            }
          }
          if (lane == 0) {
            sh.gn = g;
            sh.gktot = ktot;
            sh.gfast = fast;
            sh.sacc = gsacc;
            sh.sop = 0;
          }
        }
      }
      __syncthreads();
      if (sh.abort) break;
      const int g = sh.gn;
      if (packed) {
        const bool ok = mbar_wait_bounded(&sh.stage_bar, stage_phase, ctrl, w.timeout_ns);
        stage_phase ^= 1u;
        if (__syncthreads_or(!ok)) {
          if (tid == 0) atomicCAS(&ctrl->err, 0, SYLV_ERR_TIMEOUT);
          sh.abort = 1;
          break;
        }
      } else if constexpr (TT == 32 && sizeof(T) == 8) {
        // All of the group's global loads are issued before any shared-memory store
        // (through generic pointers the compiler cannot reorder them), so the group
        // costs one memory round trip instead of one per operand tile.  (The binary32
        // kernel has no registers to spare for it.)
        constexpr int GM = DagSmem<TT, T>::G;
        constexpr int PT = TT * TT / kThreads;  // elements per thread of one operand tile
        constexpr int LDG = DagSmem<TT, T>::LDG;
        T vl[GM][PT], vr[GM][PT];
#pragma unroll
        for (int u = 0; u < GM; ++u) {
          if (u < g) {
            const int side = sh.gside[u], prod = sh.gprod[u], kdim = sh.gk[u];
            const T* PL;
            const T* PR;
            int64_t ldl, ldr;
            if (side == 0) {  // A_ki (rows of tile k) and Y_il
              const int i = prod / I.qmax;
              PL = A + r0 + (int64_t)rb[i] * I.lda;
              ldl = I.lda;
              PR = C + rb[i] + (int64_t)c0 * I.ldc;
              ldr = I.ldc;
            } else {  // Y_kj and B_jl
              const int j = prod % I.qmax;
              PL = C + r0 + (int64_t)cb[j] * I.ldc;
              ldl = I.ldc;
              PR = B + cb[j] + (int64_t)c0 * I.ldb;
              ldr = I.ldb;
            }
#pragma unroll
            for (int e = 0; e < PT; ++e) {
              const int idx = tid + e * kThreads;
              const int r = idx % TT, kk = idx / TT;
              T v = T(0);
              if (r < mt && kk < kdim) v = side ? __ldcg(PL + r + kk * ldl) : __ldg(PL + r + kk * ldl);
              vl[u][e] = v;
              const int kk2 = idx % kdim, c = idx / kdim;
              T v2 = T(0);
              if (c < nt && idx < TT * kdim) v2 = side ? __ldg(PR + kk2 + c * ldr) : __ldcg(PR + kk2 + c * ldr);
              vr[u][e] = v2;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < GM; ++u) {
          if (u < g) {
            const int kdim = sh.gk[u];
            T* Lu = sh.L + sh.goff[u] * LDG;
            T* Ru = sh.R + sh.goff[u] * LDG;
#pragma unroll
            for (int e = 0; e < PT; ++e) {
              const int idx = tid + e * kThreads;
              if (idx < TT * kdim) {
                Lu[(idx / TT) * LDG + idx % TT] = vl[u][e];
                Ru[(idx % kdim) * LDG + idx / kdim] = vr[u][e];
              }
            }
          }
        }
      } else {
        for (int u = 0; u < g; ++u) {
          const int side = sh.gside[u], prod = sh.gprod[u], kdim = sh.gk[u];
          T* Lu = sh.L + sh.goff[u] * DagSmem<TT, T>::LDG;
          T* Ru = sh.R + sh.goff[u] * DagSmem<TT, T>::LDG;
          if (side == 0) {
            const int i = prod / I.qmax;
            stage_left<TT, T, false>(Lu, A + r0 + (int64_t)rb[i] * I.lda, I.lda, mt, kdim);
            stage_right<TT, T, true>(Ru, C + rb[i] + (int64_t)c0 * I.ldc, I.ldc, kdim, nt);
          } else {
            const int j = prod % I.qmax;
            stage_left<TT, T, true>(Lu, C + r0 + (int64_t)cb[j] * I.ldc, I.ldc, mt, kdim);
            stage_right<TT, T, false>(Ru, B + cb[j] + (int64_t)c0 * I.ldb, I.ldb, kdim, nt);
          }
        }
      }
      if (w.prio && tid == 0) {
        // A diagonal solve on this SM is on the critical path: let it have the FP64
        // pipe (bounded: at most ~200 us per group).
        const int32_t* busy = w.smbusy + sm_id();
        for (int it = 0; it < 400 && ld_volatile(busy) > 0; ++it) __nanosleep(500);
      }
      if (ROBUST && tid == 0 && !sh.gfast) {
        const int side = sh.gside[0], prod = sh.gprod[0];
        const int ep = texp[prod];
        const double yp = tnorm[prod];
        const double on = opnorm(side, prod);
        const int eta = min(sh.e_acc, ep);
        const double c = mul2(sh.nb_acc, eta - sh.e_acc);
        const double x = mul2(yp, eta - ep);
        const int z = (side == 0) ? protect_update(c, on, x, omega) : protect_update(c, x, on, omega);
        const int delta = eta + z;
        sh.sacc = delta - sh.e_acc;
        sh.sop = delta - ep;
        sh.nb_acc = mul2(sh.nb_acc, sh.sacc) + on * mul2(yp, sh.sop);
        sh.e_acc = delta;
        if (sh.sacc != 0 || sh.sop != 0) ++sh.nscale;
      }
      __syncthreads();
      if (ROBUST) {
        const int sop = sh.sop, sacc = sh.sacc;
        if (sop != 0) {  // single producer: scale its Y operand (R on the A side, L on the B side)
          T* Yop = (sh.gside[0] == 0) ? sh.R : sh.L;
          const int nel = sh.gk[0] * DagSmem<TT, T>::LDG;
          for (int idx = tid; idx < nel; idx += kThreads) Yop[idx] = mul2(Yop[idx], sop);
          __syncthreads();
        }
        if (sh.gfast == 2) {  // scaled group: each producer's Y operand to the common exponent
          constexpr int LDG = DagSmem<TT, T>::LDG;
          for (int u = 0; u < g; ++u) {
            const int so = sh.gsop[u];
            if (so == 0) continue;
            T* Yop = ((sh.gside[u] == 0) ? sh.R : sh.L) + sh.goff[u] * LDG;
            const int nel = sh.gk[u] * LDG;
            for (int idx = tid; idx < nel; idx += kThreads) Yop[idx] = mul2(Yop[idx], so);
          }
          __syncthreads();
        }
        if (sacc != 0) {
#pragma unroll
          for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < NR; ++j) {
              acc[i][j] = mul2(acc[i][j], sacc);
              acc_lo[i][j] = mul2(acc_lo[i][j], sacc);
            }
        }
      }
      if constexpr (kComp) {
        T part[MR][NR];
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
          for (int j = 0; j < NR; ++j) part[i][j] = T(0);
        if constexpr (DagSmem<TT, T>::kSplitK)
          gemm_sub_split4<TT, T>(part, sh.L, sh.R, sh.gktot, rbase, cbase, sh.kred);
        else
          gemm_sub<TT, T, MR, NR>(part, sh.L, sh.R, sh.gktot, rbase, cbase);
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
          for (int j = 0; j < NR; ++j) {  // two-sum: acc + part = t + e exactly
            const T t = acc[i][j] + part[i][j];
            const T bp = t - acc[i][j];
            const T e = (acc[i][j] - (t - bp)) + (part[i][j] - bp);
            acc[i][j] = t;
            acc_lo[i][j] += e;
          }
      } else {
        gemm_sub<TT, T, MR, NR>(acc, sh.L, sh.R, sh.gktot, rbase, cbase);
      }
      __syncthreads();
      q += g;
    }
    if (sh.abort) break;

    // ---- diagonal problem A_kk Z + Z B_ll = beta Y_kl
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) sh.Y[(rbase + i) + (cbase + j) * LDY] = acc[i][j] + acc_lo[i][j];
    for (int idx = tid; idx < TT * TT; idx += kThreads) {
      const int r = idx % TT, c = idx / TT;
      sh.L[r + c * LDY] = (r < mt && c < mt && r <= c + 1) ? __ldg(&A[(r0 + r) + (int64_t)(r0 + c) * I.lda]) : T(0);
      sh.R[r + c * LDY] =
          (!I.nob && r < nt && c < nt && r <= c + 1) ? __ldg(&B[(c0 + r) + (int64_t)(c0 + c) * I.ldb]) : T(0);
    }
    if (w.prio && tid == 0) atomicAdd(w.smbusy + sm_id(), 1);
    __syncthreads();
    diag_solve<TT, T, ROBUST>(sh, mt, nt, omega, st->smin, fact, factp, I.nob != 0);
    if (w.prio && tid == 0) atomicSub(w.smbusy + sm_id(), 1);

    // ---- infinity norm of the final tile (binary64 row sums), write back, publish.
    // A warp per row, lanes across the columns and a shuffle tree, so the sum is a
    // short dependency chain on the FP64 pipe; the maximum is taken on the bit
    // patterns of the non-negative sums, so a NaN row still reaches the check below.
    if (tid == 0) sh.umax = 0ull;
    __syncthreads();
    tile_norm_max<TT, T>(sh, mt, nt);
    for (int idx = tid; idx < mt * nt; idx += kThreads) {
      const int r = idx % mt, c = idx / mt;
      C[(r0 + r) + (int64_t)(c0 + c) * I.ldc] = sh.Y[r + c * LDY];
    }
    if (packed) {
      // The tile as a left operand (column-major, YL[c][r]) and as a right operand
      // (row-major, YR[r][c]), zero-padded, for its consumers' bulk copies; the proxy
      // fence orders these generic stores before the async-proxy reads that follow
      // the flag.
      constexpr int LDG = DagSmem<TT, T>::LDG;
      T* yl = reinterpret_cast<T*>(w.pack + pack_yl(I, k, l) * w.pack_slot);
      T* yr = reinterpret_cast<T*>(w.pack + pack_yr(I, k, l) * w.pack_slot);
      for (int idx = tid; idx < TT * LDG; idx += kThreads) {
        const int kk = idx / LDG, x = idx % LDG;
        yl[idx] = (x < mt && kk < nt) ? sh.Y[x + kk * LDY] : T(0);
        yr[idx] = (x < nt && kk < mt) ? sh.Y[kk + x * LDY] : T(0);
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      const double nrm = __longlong_as_double(static_cast<long long>(sh.umax));
      const int e = ROBUST ? sh.e_acc + sh.e_diag : 0;
      texp[task.tile] = e;
      tnorm[task.tile] = nrm;
      __threadfence();
      st_release64(&tflag[task.tile], tile_word(e, nrm));
      // The equation's status words are read only after the kernel, so their atomics
      // follow the release instead of delaying it.
      int fl = sh.flags;
      if (!(nrm <= 1.7976931348623157e308)) fl |= kFlagNonfiniteOut;
      if (fl) atomicOr(&st->flags, fl);
      if (ROBUST) {
        atomicMin(&st->minexp, e);
        if (sh.nscale) atomicAdd(&st->nscale, sh.nscale);
      }
    }
    __syncthreads();
  }
}

}  // namespace sylv
