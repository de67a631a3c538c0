// sylv_oz.cuh -- the first residual of the refinement, R = C - (A X + X B), to
// binary64 accuracy on the bf16 tensor cores (tcgen05, sm_103a).
//
// Error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", 2012, written here for bf16 operands with
// binary32 accumulation).  Every row r of the left operand gets a power of two
// 2^e_r above its largest magnitude, and every value v of the row is written as
//     v = 2^e_r * sum_{s=1..S} a_s 2^(-8s) + (error below 2^(e_r - 8S)),
// with integer slices a_1 in [-256, 256] and a_s in [-128, 128] for s > 1 (each an
// exact bf16).  The right operand is split the same way per column.  A product of
// two slices is an integer of magnitude <= 2^16, so a sum of 256 of them is an
// exact integer below 2^24 and the tensor core's binary32 accumulation of it is
// exact: the kernel accumulates chunks of 256 in TMEM, converts each chunk to
// int32 (exact) and sums chunks in int32, pairs of equal weight 2^(-8(s+t))
// together; every 64 chunks or at the end of a weight it adds the integer, scaled
// by 2^(e_r + e_c - 8(s+t)), into a binary64 accumulator.  Pairs with s + t > S + 1
// are dropped: with S = 7 they weigh below 2^-56 of (row maximum) x (column maximum)
// per product term, as do the truncated slices; the binary64 sums of the ~14
// flushes per element add rounding below 2^-49 of the products' magnitude.  The
// guarantee is relative to the row and column maxima (normwise): with balanced rows
// and columns it is about 2^-48 componentwise (|A||X| + |X||B|), like the
// double-float kernel it replaces; rows dominated by one large entry (a heavy
// diagonal) keep correspondingly fewer bits of their small entries.
//
// Layouts.  Operand slices are stored pre-tiled in the canonical no-swizzle K-major
// layout of tcgen05: a tile is R rows x 64 K elements (R = 128 for the left
// operand, 64 for the right), made of 8 x 8 core matrices (8 rows of 16 bytes,
// 128 contiguous bytes), core matrix (row/8, k/8) at index (row/8)*8 + k/8.  A tile
// is contiguous, so one 1D bulk copy (cp.async.bulk) moves it into shared memory.
// Products: A X uses A (rows of A, K = columns, quasi-upper mask) and X by columns
// (N = columns of X, K = rows); X B uses X by rows (K = columns of X) and B by
// columns (N = columns of B, K = rows, quasi-upper mask).
//
// The same kernel with only the pairs s + t <= 6 (dropped terms below 2^-40 of the
// maxima) serves the later residuals of the refinement, R_k = R_{k-1} - (A D + D B),
// in place (C = R): the correction D is small, and its product needs only to be
// well below the next residual.
//
// The GEMM kernel: one CTA per 128 x 64 tile of R, 192 threads.  Warp 4 issues the
// bulk copies into a 4-stage shared-memory ring (mbarriers with transaction
// counts), one thread of warp 5 issues the MMAs (M = 128, N = 64, K = 16) into two
// TMEM accumulators used alternately per chunk, and warps 0-3 (one TMEM lane
// quarter each, one row of the tile per thread) take each finished chunk out of
// TMEM.  Every wait is bounded; a timeout records SYLV_ERR_TIMEOUT.
#pragma once

#include <cuda_bf16.h>

#include "sylv_internal.cuh"

namespace sylv {
namespace oz {

constexpr int kSlices = 7;             // 8-bit slices per operand (56 bits below the maximum)
constexpr int kMaxW = kSlices + 1;     // binary64 residual: pairs (s, t), 1-based, with s + t <= kMaxW
constexpr int kMaxW32 = 6;             // products for the binary32 recurrence: s + t <= 6 (40 bits)
constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kLeadW = 4;              // weights 2..4 are accumulated exactly (chunked)
constexpr int kLeadStages = 6;         // 6 K blocks of 32 per exact binary32 chunk (< 2^24, see below)
constexpr int kFlushLead = 64;         // chunks per int32 sum: 64 * 2^24 = 2^30 < 2^31
constexpr int NST = 2;                 // shared-memory stages (all slices of one K block each)
constexpr int kTileA = BM * BK;        // bf16 elements of a left-operand tile (8 KB)
constexpr int kTileB = BN * BK;        // of a right-operand tile (4 KB)
constexpr int kEpiWarps = 8;           // two per TMEM lane quarter, 32 columns each
constexpr int kThreads = 32 * (kEpiWarps + 2);

struct Smem {
  __nv_bfloat16 a[NST][kSlices][kTileA];
  __nv_bfloat16 b[NST][kSlices][kTileB];
  int ecol[2][BN];
  unsigned long long full[NST], empty[NST], accfull, accempty;
  uint32_t tmem;
};

// One operand view: element (r, k) of the operand is src[r * rs + k * ks] within
// rows x kdim; mask 1 keeps r <= k + 1 (A), mask 2 keeps k <= r + 1 (B as columns).
struct View {
  const double* src;
  int64_t rs, ks;
  int64_t rows, kdim;
  int mask;
};

// Tiled operand: RB row blocks of R rows, KB blocks of 64 K; slice s at s * slice_elems.
struct Packed {
  __nv_bfloat16* p;
  int* e;  // per-row exponent (rows padded to RB * R)
  int64_t RB, KB;
  int R;
  __host__ __device__ int64_t slice_elems() const { return RB * KB * static_cast<int64_t>(R) * BK; }
};

__device__ __forceinline__ double view_at(const View& v, int64_t r, int64_t k) {
  if (r >= v.rows || k >= v.kdim) return 0.0;
  if (v.mask == 1 && r > k + 1) return 0.0;
  if (v.mask == 2 && k > r + 1) return 0.0;
  return v.src[r * v.rs + k * v.ks];
}

// Per-row exponent: smallest e with max_k |op(r, k)| < 2^e (0 for a zero row).
// One warp per row, lanes over K.
__global__ void k_oz_rowexp(View v, int* e, int64_t rows_padded, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = wid; r < rows_padded; r += nw) {
    unsigned long long mx = 0;
    if (r < v.rows)
      for (int64_t k = lane; k < v.kdim; k += 32) {
        const unsigned long long b =
            static_cast<unsigned long long>(__double_as_longlong(view_at(v, r, k))) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = u > mx ? u : mx;
    }
    if (lane == 0) e[r] = mx ? static_cast<int>((mx >> 52) & 0x7ff) - 1022 : 0;
  }
}

// Slices of every element, one block per packed tile: the tile is read along its
// contiguous dimension into shared memory (rows when rs == 1, else K), then each
// thread takes positions of the packed layout and writes all kSlices slices of each.
__global__ void __launch_bounds__(256) k_oz_split(View v, Packed P, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  __shared__ double tile[BM * (BK + 1)];
  const int64_t per = P.slice_elems();
  const int tsz = P.R * BK;
  const bool rcontig = v.rs == 1;
  for (int64_t t = blockIdx.x; t < P.RB * P.KB; t += gridDim.x) {
    const int64_t r0 = (t / P.KB) * P.R, k0 = (t % P.KB) * BK;
    __syncthreads();  // the previous tile's reads are done
    for (int idx = threadIdx.x; idx < tsz; idx += blockDim.x) {
      const int r = rcontig ? idx % P.R : idx / BK;
      const int kk = rcontig ? idx / P.R : idx % BK;
      tile[r * (BK + 1) + kk] = view_at(v, r0 + r, k0 + kk);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < tsz; o += blockDim.x) {
      const int cm = o >> 6, w = o & 63;  // core matrix (rr/8) * (BK/8) + kk/8, then row-major 8 x 8
      const int rr = (cm / (BK / 8)) * 8 + (w >> 3), kk = (cm % (BK / 8)) * 8 + (w & 7);
      const double x = tile[rr * (BK + 1) + kk];
      double u = (x == 0.0) ? 0.0 : mul2(x, 8 - P.e[r0 + rr]);  // |u| < 256
      const int64_t idx = t * tsz + o;
#pragma unroll
      for (int s = 0; s < kSlices; ++s) {
        const double q = rint(u);
        P.p[idx + s * per] = __float2bfloat16_rn(static_cast<float>(q));  // exact: |q| <= 256, an integer
        u = (u - q) * 256.0;                                              // exact
      }
    }
  }
}

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
// Bounded wait for the phase of the given parity; false on timeout or when another
// role recorded an error.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, const int* err, long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63) {
      if (ld_volatile(err)) return false;
      if (static_cast<long long>(global_ns() - t0) > timeout_ns) return false;
    }
  }
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
// Shared-memory matrix descriptor, no swizzle: core matrices LBO bytes apart along
// K and SBO bytes apart along M/N; bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: binary32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
                            (static_cast<uint32_t>(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtm),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(ta));
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The two products of one launch: left operands (R = 128) and right operands (R = 64).
// Row panels per group of the output-tile order (8 x 19 panels resident at once).
constexpr int kGroupRows = 8;

struct Gemm {
  Packed a[2];
  Packed b[2];
};

// K blocks of product p for output rows [i0, i0+128) and columns [j0, j0+64): A X
// reads A[i, k] for k >= i - 1; X B reads B[k, j] for k <= j + 1.
__device__ __forceinline__ void kb_range(int p, const Gemm& g, int64_t i0, int64_t j0, int& lo, int& hi) {
  if (p == 0) {
    lo = i0 > 0 ? static_cast<int>((i0 - 1) / BK) : 0;
    hi = static_cast<int>(g.a[0].KB);
  } else {
    lo = 0;
    hi = static_cast<int>(min(g.a[1].KB, (j0 + BN) / BK + 1));
  }
}

// Exactness of the leading weights.  Per K block of 32, weight 2 (pair (1,1)) adds at
// most 32 * 2^16 = 2^21 in magnitude, weight 3 (pairs (1,2), (2,1)) 2 * 32 * 2^15 =
// 2^21, weight 4 ((1,3), (3,1), (2,2)) 32 * (2^15 + 2^15 + 2^14) < 2^21.33; six blocks
// stay below 2^24, so those accumulators are taken out of TMEM exactly every six
// blocks (integers, exact in binary32).  Weights >= 5 are accumulated over the whole
// K range in binary32: their rounding is below 2^-24 of a sum that is itself below
// 2^-24 of the leading term, so below 2^-48 of the result.
//
// The kernel.  One CTA per 128 x 64 tile of R; warp 8 loads, one thread of warp 9
// issues the MMAs, warps 0-7 drain TMEM (warp w: TMEM lanes 32 (w & 3).., tile
// columns 32 (w >> 2)..).  Per K block a stage holds all slices of both operands,
// and every slice pair of weight <= maxw goes into the accumulator of its weight
// (TMEM columns 64 (w - 2)..).  R starts as C and every flush subtracts its terms.
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_gemm(Gemm g, int maxw, const double* C, int64_t ldc, double* R, int64_t ldr, int64_t m, int64_t n,
              unsigned long long* rmax, int* err, long long timeout_ns, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& sh = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Output tiles in L2-friendly order: the launch runs through groups of kGroupRows
  // row panels, column panels fastest within a group, so that the CTAs resident at
  // once share a few row panels of A (and of X) and a set of column panels instead
  // of streaming every row panel's slices through L2 again for each column wave.
  int mb, nb;
  {
    const int MBt = gridDim.x, NBt = gridDim.y;
    const int id = blockIdx.x + MBt * blockIdx.y;
    const int gsize = kGroupRows * NBt;
    const int grp = id / gsize, in = id - grp * gsize;
    const int rows = min(kGroupRows, MBt - grp * kGroupRows);
    mb = grp * kGroupRows + in % rows;
    nb = in / rows;
  }
  const int64_t i0 = static_cast<int64_t>(mb) * BM, j0 = static_cast<int64_t>(nb) * BN;
  const int smax = min(kSlices, maxw - 1);  // slices in use

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    mbar_init(&sh.accfull, 1);
    mbar_init(&sh.accempty, 32 * kEpiWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 2 * BN) sh.ecol[tid / BN][tid % BN] = g.b[tid / BN].e[static_cast<int64_t>(nb) * BN + tid % BN];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = sh.tmem;

  if (warp == kEpiWarps) {
    // ---- loads: all slices in use of one K block per stage
    if (lane == 0) {
      int gs = 0;
      bool ok = true;
      const uint32_t bytes = static_cast<uint32_t>(smax) * (kTileA + kTileB) * 2;
      for (int p = 0; p < 2 && ok; ++p) {
        int lo, hi;
        kb_range(p, g, i0, j0, lo, hi);
        const Packed& A = g.a[p];
        const Packed& B = g.b[p];
        const __nv_bfloat16* ab = A.p + (static_cast<int64_t>(mb) * A.KB) * kTileA;
        const __nv_bfloat16* bb = B.p + (static_cast<int64_t>(nb) * B.KB) * kTileB;
        for (int kb = lo; kb < hi; ++kb, ++gs) {
          const int st = gs & 1;
          if (!mbar_wait(&sh.empty[st], ((gs >> 1) & 1) ^ 1, err, timeout_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sh.full[st], bytes);
          for (int sl = 0; sl < smax; ++sl) {
            bulk_g2s(sh.a[st][sl], ab + sl * A.slice_elems() + static_cast<int64_t>(kb) * kTileA, kTileA * 2,
                     &sh.full[st]);
            bulk_g2s(sh.b[st][sl], bb + sl * B.slice_elems() + static_cast<int64_t>(kb) * kTileB, kTileB * 2,
                     &sh.full[st]);
          }
        }
      }
      if (!ok) atomicCAS(err, 0, SYLV_ERR_TIMEOUT);
    }
  } else if (warp == kEpiWarps + 1) {
    // ---- MMAs
    if (lane == 0) {
      int gs = 0, ev = 0, pend = -1;  // pend: event whose drain must end before the accumulators it frees are reused
      bool pend_all = false, ok = true;
      for (int p = 0; p < 2 && ok; ++p) {
        int lo, hi;
        kb_range(p, g, i0, j0, lo, hi);
        unsigned written = 0;  // weights written since their last drain
        int since = 0;
        for (int kb = lo; kb < hi && ok; ++kb, ++gs) {
          const int st = gs & 1;
          if (!mbar_wait(&sh.full[st], (gs >> 1) & 1, err, timeout_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (pend >= 0 && pend_all) {  // a product ended: every accumulator is being drained
            if (!mbar_wait(&sh.accempty, pend & 1, err, timeout_ns)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            pend = -1;
          }
          for (int pass = 0; pass < 2; ++pass) {  // weights >= 5 first, then the leading ones
            if (pass == 1 && pend >= 0) {  // the leading accumulators are being drained
              if (!mbar_wait(&sh.accempty, pend & 1, err, timeout_ns)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              pend = -1;
            }
            for (int w = pass ? 2 : kLeadW + 1; w <= (pass ? kLeadW : maxw); ++w)
              for (int sl = max(1, w - smax); sl <= min(smax, w - 1); ++sl) {
                const int t = w - sl;
                const uint32_t aa = su32(sh.a[st][sl - 1]), ba = su32(sh.b[st][t - 1]);
                const uint32_t dtm = tbase + static_cast<uint32_t>((w - 2) * BN);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                  const bool acc = ((written >> w) & 1u) != 0;
                  umma(dtm, sdesc(aa + kk * 256, 128, (BK / 8) * 128), sdesc(ba + kk * 256, 128, (BK / 8) * 128),
                       acc ? 1u : 0u);
                  written |= 1u << w;
                }
              }
          }
          if (!ok) break;
          umma_commit(&sh.empty[st]);
          ++since;
          const bool last = kb == hi - 1;
          if (last || since == kLeadStages) {
            umma_commit(&sh.accfull);
            pend = ev++;
            pend_all = last;
            written = last ? 0u : (written & ~((1u << (kLeadW + 1)) - 1u));
            since = 0;
          }
        }
      }
      if (!ok) atomicCAS(err, 0, SYLV_ERR_TIMEOUT);
    }
  } else {
    // ---- drain: row 32 (warp & 3) + lane, columns 32 (warp >> 2)..
    const int row = 32 * (warp & 3) + lane;
    const int cb0 = 32 * (warp >> 2);
    const int64_t gi = i0 + row;
    const uint32_t tl = tbase + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
    if (gi < m && C != R)
      for (int j = 0; j < 32; ++j) {
        const int64_t gj = j0 + cb0 + j;
        if (gj < n) R[gi + gj * ldr] = C[gi + gj * ldc];
      }
    int iacc[kLeadW - 1][32];
#pragma unroll
    for (int a = 0; a < kLeadW - 1; ++a)
#pragma unroll
      for (int j = 0; j < 32; ++j) iacc[a][j] = 0;
    int ev = 0;
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
      int lo, hi;
      kb_range(p, g, i0, j0, lo, hi);
      const int erow = g.a[p].e[gi];
      const int nst = hi - lo;
      const int nlead = (nst - 1) / kLeadStages;  // drains of the leading weights before the last
      int nacc = 0;
      for (int d = 0; d <= nlead && ok; ++d, ++ev) {
        const bool last = d == nlead;
        if (!mbar_wait(&sh.accfull, ev & 1, err, timeout_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int a = 0; a < kLeadW - 1; ++a) {
          uint32_t v0[16], v1[16];
          tmem_ld16(tl + static_cast<uint32_t>(a * BN + cb0), v0);
          tmem_ld16(tl + static_cast<uint32_t>(a * BN + cb0 + 16), v1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            iacc[a][j] += __float2int_rn(__uint_as_float(v0[j]));
            iacc[a][16 + j] += __float2int_rn(__uint_as_float(v1[j]));
          }
        }
        ++nacc;
        const bool flush = last || nacc == kFlushLead;  // the same in every lane (TMEM loads are warp-collective)
        if (flush) {
          // R -= 2^(e_row + e_col) * (sum over weights w of 2^(-8w) * sum_w), smallest weights first
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            double dsum[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) dsum[j] = 0.0;
            if (last)
              for (int w = maxw; w > kLeadW; --w) {
                uint32_t v[16];
                tmem_ld16(tl + static_cast<uint32_t>((w - 2) * BN + cb0 + 16 * h), v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const float f = __uint_as_float(v[j]);
                  if (f != 0.0f)
                    dsum[j] += mul2(static_cast<double>(f), erow + sh.ecol[p][cb0 + 16 * h + j] - 8 * w);
                }
              }
#pragma unroll
            for (int a = kLeadW - 2; a >= 0; --a)
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (iacc[a][16 * h + j] != 0)
                  dsum[j] += mul2(static_cast<double>(iacc[a][16 * h + j]),
                                  erow + sh.ecol[p][cb0 + 16 * h + j] - 8 * (a + 2));
            if (gi < m)
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int64_t gj = j0 + cb0 + 16 * h + j;
                if (gj < n) R[gi + gj * ldr] -= dsum[j];
              }
          }
        }
        if (flush) {
#pragma unroll
          for (int a = 0; a < kLeadW - 1; ++a)
#pragma unroll
            for (int j = 0; j < 32; ++j) iacc[a][j] = 0;
          nacc = 0;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh.accempty);
      }
    }
    if (!ok) atomicCAS(err, 0, SYLV_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
  if (ld_volatile(err) || !rmax) return;
  // ---- max |R| of the tile
  if (warp < kEpiWarps) {
    const int row = 32 * (warp & 3) + lane;
    const int cb0 = 32 * (warp >> 2);
    const int64_t gi = i0 + row;
    double mx = 0.0;
    if (gi < m)
      for (int j = 0; j < 32; ++j) {
        const int64_t gj = j0 + cb0 + j;
        if (gj < n) mx = fmax(mx, fabs(R[gi + gj * ldr]));
      }
    mx = warp_max(mx);
    if (lane == 0) atomic_max_nonneg(rmax, mx);
  }
}

}  // namespace oz
}  // namespace sylv
