// sylv_oz.cuh -- the first residual of the refinement, R = C - (A X + X B), to
// binary64 accuracy on the bf16 tensor cores (tcgen05, sm_103a).
//
// Error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", 2012, written here for bf16 operands with
// binary32 accumulation).  Every row r of the left operand gets a power of two
// 2^e_r above its largest magnitude, and every value v of the row is written as
//     v = 2^e_r * sum_{s=1..S} a_s 2^(-8s) + (error below 2^(e_r - 8S)),
// with integer slices a_1 in [-256, 256] and a_s in [-128, 128] for s > 1, stored
// pre-scaled as the exact bf16 values a_s 2^(-8(s-1)).  The right operand is split
// the same way per column.  A product of two integer slices has magnitude <= 2^16,
// so a sum of 256 of them is an exact integer below 2^24 and the tensor core's
// binary32 accumulation of it is exact (a power-of-two scale changes nothing): the
// kernel accumulates the pairs of each of the three leading weights s + t = 2, 3, 4
// in chunks of 192 in TMEM, converts each chunk to integers (exact) and sums the
// chunks in one int64 per element; each smaller weight has a binary32 accumulator
// of its own; at the end of a product both go, scaled by 2^(e_r + e_c - 32), into R
// in binary64.  Pairs with s + t > S + 1 are dropped: with S = 7 they weigh below
// 2^-56 of (row maximum) x (column maximum) per product term, as does the rounding
// of the elements to 56 bits; the binary32 sums of the smaller weights are rounded
// at 2^-24 of terms that are themselves below 2^-24 of the leading ones, and the two
// binary64 updates of each element (one per product) round at 2^-53.  The
// guarantee is relative to the row and column maxima (normwise): with balanced rows
// and columns it is about 2^-48 componentwise (|A||X| + |X||B|), like the
// double-float kernel it replaces; rows dominated by one large entry (a heavy
// diagonal) keep correspondingly fewer bits of their small entries.
//
// Layouts.  Operand slices are stored pre-tiled in the canonical no-swizzle K-major
// layout of tcgen05: a tile is R rows x 16 K elements (R = 128 for the left
// operand, 64 for the right), made of 8 x 8 core matrices (8 rows of 16 bytes,
// 128 contiguous bytes), core matrix (row/8, k/8) at index (row/8)*2 + k/8.  A tile
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
// The GEMM kernel: one CTA per 128 x 64 tile of R, 320 threads (details at the
// kernel).  Every wait is bounded; a timeout records SYLV_ERR_TIMEOUT.
#pragma once

#include <cuda_bf16.h>

#include "sylv_internal.cuh"

namespace sylv {
namespace oz {

constexpr int kSlices = 7;             // 8-bit slices per operand (56 bits below the maximum)
constexpr int kMaxW = kSlices + 1;     // binary64 residual: pairs (s, t), 1-based, with s + t <= kMaxW
constexpr int kMaxW32 = 6;             // products for the binary32 recurrence: s + t <= 6 (40 bits)
constexpr int BM = 128, BN = 64, BK = 16;
constexpr int kLeadW = 4;              // weights 2..4 are accumulated exactly (chunked)
constexpr int kLeadStages = 12;        // 12 K blocks of 16 per exact binary32 chunk (< 2^24, see below)
constexpr int NST = 5;                 // shared-memory stages (all slices of one K block each)
constexpr int kTileA = BM * BK;        // bf16 elements of a left-operand tile (4 KB)
constexpr int kTileB = BN * BK;        // of a right-operand tile (2 KB)
constexpr int kEpiWarps = 8;           // two per TMEM lane quarter, 32 columns each
constexpr int kThreads = 32 * (kEpiWarps + 2);


// One operand view: element (r, k) of the operand is src[r * rs + k * ks] within
// rows x kdim; mask 1 keeps r <= k + 1 (A), mask 2 keeps k <= r + 1 (B as columns).
struct View {
  const double* src;
  int64_t rs, ks;
  int64_t rows, kdim;
  int mask;
};

// Tiled operand: RB row blocks of R rows, KB blocks of BK along K; slice s at s * slice_elems.
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
__device__ __forceinline__ void oz_rowexp(const View& v, int* e, int64_t rows_padded) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = wid; r < rows_padded; r += nw) {
    unsigned long long mx = 0;
    if (r < v.rows)
#pragma unroll 4
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
__global__ void k_oz_rowexp(View v, int* e, int64_t rows_padded, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  oz_rowexp(v, e, rows_padded);
}

// round(x * 2^(56 - e)) as an integer, for |x| < 2^e: the element on the grid of
// its row's 56 bits (|result| <= 2^56), from the bits of x alone.
__device__ __forceinline__ long long fixed56(double x, int e) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  unsigned long long M = b & ((1ull << 52) - 1);
  if (E != 0) M |= 1ull << 52;
  const int sh = (E != 0 ? E : 1) - 1019 - e;  // x = +-M 2^(E - 1075)
  long long v;
  if (sh >= 0)
    v = static_cast<long long>(M << sh);  // M 2^sh < 2^56
  else if (sh > -60)
    v = static_cast<long long>((M + (1ull << (-sh - 1))) >> (-sh));
  else
    v = 0;
  return (b >> 63) ? -v : v;
}

// Slices of every element, one block per packed tile: the tile is read along its
// contiguous dimension into shared memory (rows when rs == 1, else K), then each
// thread takes positions of the packed layout and writes all kSlices slices of each.
// In integers: V = round(x 2^(56 - e_r)), then signed base-256 digits from the top,
// q_1 = round(V / 2^48), V -= q_1 2^48, q_2 = round(V / 2^40), ..., q_7 = V, so that
// |q_1| <= 256, |q_s| <= 128 and x = 2^(e_r - 8) sum_s q_s 2^(-8(s-1)) to within
// 2^(e_r - 57).  Slice s is stored pre-scaled, q_s 2^(-8(s-1)) (exact in bf16), so
// that a product of slices s and t carries its weight 2^(-8(s+t-2)) relative to
// the leading pair.  Infinities and NaN give NaN slices.
__device__ __forceinline__ void oz_split(const View& v, const Packed& P, double* tile) {
  const int64_t per = P.slice_elems();
  const int tsz = P.R * BK;
  const bool rcontig = v.rs == 1;
  for (int64_t t = blockIdx.x; t < P.RB * P.KB; t += gridDim.x) {
    const int64_t r0 = (t / P.KB) * P.R, k0 = (t % P.KB) * BK;
    // Tiles the products never read (kb_range): A's K blocks left of its row panel's
    // diagonal, B's (as columns) beyond its column panel's; all masked zeros.
    if ((v.mask == 1 && r0 > 0 && k0 / BK < (r0 - 1) / BK) || (v.mask == 2 && k0 / BK > (r0 + P.R) / BK)) continue;
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
      const bool finite = ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
      long long V = finite ? fixed56(x, P.e[r0 + rr]) : 0;
      const int64_t idx = t * tsz + o;
      if (finite && V == 0) {  // zeros (padding, masked entries): every slice is zero
#pragma unroll
        for (int s = 0; s < kSlices; ++s) P.p[idx + s * per] = __float2bfloat16_rn(0.0f);
        continue;
      }
#pragma unroll
      for (int s = 0; s < kSlices; ++s) {
        const int sh = 8 * (kSlices - 1 - s);
        long long q = V;
        if (sh > 0) {
          q = (V + (1ll << (sh - 1))) >> sh;
          V -= q << sh;
        }
        const float scale = __int_as_float((127 - 8 * s) << 23);  // 2^(-8s)
        const float f = finite ? static_cast<float>(static_cast<int>(q)) * scale : __int_as_float(0x7fc00000);
        P.p[idx + s * per] = __float2bfloat16_rn(f);  // exact: an integer of at most 9 bits times 2^(-8s)
      }
    }
  }
}
__global__ void __launch_bounds__(256) k_oz_split(View v, Packed P, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  __shared__ double tile[BM * (BK + 1)];
  oz_split(v, P, tile);
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
// K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128; N a multiple of 64 up to 256).
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(BM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
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
  int dense;  // 1: one unstructured product a[0] b[0]^T over all of K (b[1] unused)
};

struct Smem {
  __nv_bfloat16 a[NST][kSlices][kTileA];
  __nv_bfloat16 b[NST][kSlices][kTileB];
  int ecol[2][BN];
  unsigned long long full[NST], empty[NST], accfull, accempty;
  uint32_t tmem;
  Gemm g;  // batched launches: the tile's equation
};

// K blocks of product p for output rows [i0, i0+128) and columns [j0, j0+64): A X
// reads A[i, k] for k >= i - 1; X B reads B[k, j] for k <= j + 1.  A dense product
// reads every K block, and there is no second product.
__device__ __forceinline__ void kb_range(int p, const Gemm& g, int64_t i0, int64_t j0, int& lo, int& hi) {
  if (g.dense) {
    lo = 0;
    hi = p == 0 ? static_cast<int>(g.a[0].KB) : 0;
  } else if (p == 0) {
    lo = i0 > 0 ? static_cast<int>((i0 - 1) / BK) : 0;
    hi = static_cast<int>(g.a[0].KB);
  } else {
    lo = 0;
    hi = static_cast<int>(min(g.a[1].KB, (j0 + BN) / BK + 1));
  }
}

// Exactness of the leading weights.  Per K block of 16, weight 2 (pair (1,1)) adds at
// most 16 * 2^16 = 2^20 in magnitude, weight 3 (pairs (1,2), (2,1)) 2 * 16 * 2^15 =
// 2^20, weight 4 ((1,3), (3,1), (2,2)) 16 * (2^15 + 2^15 + 2^14) = 1310720, counted
// as integers; twelve blocks stay below 2^24 (15728640).  With the pre-scaled slices
// the accumulator of weight w holds its integer sum times 2^(-8(w-2)), a power of two
// that keeps every partial sum exact in binary32, so those three accumulators are
// taken out of TMEM exactly every twelve blocks.  Each weight >= 5 has its own
// binary32 accumulator over the whole K range: its rounding is below 2^-24 of a sum
// that is itself below 2^-24 of the leading term, so below 2^-48 of the result.
// (One accumulator shared by all weights >= 5 loses more: the tensor core adds the
// small weights' products to a running sum up to 2^24 times larger, and at K = 300
// the error measured 2^-40 of the leading term.)

// Descriptor steps (16-byte units): one slice tile within a stage, one stage.
constexpr uint64_t kDescSliceA = kTileA * 2 / 16, kDescSliceB = kTileB * 2 / 16;
constexpr uint64_t kDescStageA = kSlices * kDescSliceA, kDescStageB = kSlices * kDescSliceB;
static_assert(BK == 16, "one MMA (K = 16) per slice pair and K block");

// The slice pairs of one staged K block whose weight is at most kLeadW (LEAD) or
// above it.  For a left slice s the pairs (s, t) with consecutive t have consecutive
// weights s + t, whose accumulators are adjacent in TMEM (64 columns each), and
// their right slices are adjacent in the stage (one 64-row tile each, 2 KB apart,
// which is 8 core-matrix rows at the 256-byte row stride), so one MMA with
// N = 64 x (number of t) computes all of them and reads the left tile once.  That is
// 10 MMAs per K block instead of 28 for the binary64 residual.  The group of s = 1
// reaches every weight of its part (2..kLeadW, or kLeadW+1..MAXW), so it alone
// carries acc0 (overwrite when 0) and is issued first.  Fully unrolled: addresses
// and instruction descriptors are the stage's bases plus constants (a shared address
// below 256 KB never carries out of the descriptor's 14-bit address field).
template <bool LEAD, int MAXW, int SMAX>
__device__ __forceinline__ void issue_part(uint32_t tbase, uint64_t da, uint64_t db, uint32_t acc0) {
  static_assert(SMAX == MAXW - 1 && SMAX >= kLeadW - 1, "the group of s = 1 spans every weight of its part");
#pragma unroll
  for (int sl = 1; sl <= SMAX; ++sl) {
    const int wlo = LEAD ? sl + 1 : (sl + 1 > kLeadW + 1 ? sl + 1 : kLeadW + 1);
    const int whi = LEAD ? (sl + SMAX < kLeadW ? sl + SMAX : kLeadW) : (sl + SMAX < MAXW ? sl + SMAX : MAXW);
    if (whi < wlo) continue;
    const int tlo = wlo - sl, cnt = whi - wlo + 1;
    umma(tbase + static_cast<uint32_t>((wlo - 2) * BN), da + (sl - 1) * kDescSliceA, db + (tlo - 1) * kDescSliceB,
         idesc_n(cnt * BN), sl == 1 ? acc0 : 1u);
  }
}
static_assert(kMaxW - kLeadW <= 4 && kLeadW - 1 <= 4, "N = 64 x (weights per MMA) <= 256");

// The kernel.  One CTA per 128 x 64 tile of R; warp 8 loads, one thread of warp 9
// issues the MMAs, warps 0-7 drain TMEM (warp w: TMEM lanes 32 (w & 3).., tile
// columns 32 (w >> 2)..).  Per K block a stage holds all slices of both operands,
// and every slice pair of weight <= MAXW goes into the accumulator of its weight
// (TMEM columns 64 (w - 2)..).  R starts as C and the end of each product subtracts
// its terms.
// One 128 x 64 output tile (row panel mb, column panel nb) of R = C - (A X + X B)
// (or of R -= L Q^T in the dense form); the whole CTA.
template <int MAXW>
__device__ __forceinline__ void oz_tile(Smem& sh, const Gemm& g, const double* C, int64_t ldc, double* R, int64_t ldr,
                                        int64_t m, int64_t n, unsigned long long* rmax, int* err,
                                        long long timeout_ns, int mb, int nb) {
  constexpr int SMAX = MAXW - 1 < kSlices ? MAXW - 1 : kSlices;  // slices in use
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = static_cast<int64_t>(mb) * BM, j0 = static_cast<int64_t>(nb) * BN;

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
      int st = 0;
      uint32_t ph = 0;
      bool ok = true;
      constexpr uint32_t bytes = static_cast<uint32_t>(SMAX) * (kTileA + kTileB) * 2;
      for (int p = 0; p < 2 && ok; ++p) {
        int lo, hi;
        kb_range(p, g, i0, j0, lo, hi);
        const Packed& A = g.a[p];
        const Packed& B = g.b[p];
        const __nv_bfloat16* ab = A.p + (static_cast<int64_t>(mb) * A.KB) * kTileA;
        const __nv_bfloat16* bb = B.p + (static_cast<int64_t>(nb) * B.KB) * kTileB;
        for (int kb = lo; kb < hi; ++kb) {
          if (!mbar_wait(&sh.empty[st], ph ^ 1, err, timeout_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sh.full[st], bytes);
#pragma unroll
          for (int sl = 0; sl < SMAX; ++sl) {
            bulk_g2s(sh.a[st][sl], ab + sl * A.slice_elems() + static_cast<int64_t>(kb) * kTileA, kTileA * 2,
                     &sh.full[st]);
            bulk_g2s(sh.b[st][sl], bb + sl * B.slice_elems() + static_cast<int64_t>(kb) * kTileB, kTileB * 2,
                     &sh.full[st]);
          }
          if (++st == NST) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) atomicCAS(err, 0, SYLV_ERR_TIMEOUT);
    }
  } else if (warp == kEpiWarps + 1) {
    // ---- MMAs
    if (lane == 0) {
      int st = 0, ev = 0, pend = -1;  // pend: event whose drain must end before the accumulators it frees are reused
      uint32_t ph = 0;
      bool pend_all = false, ok = true;
      const uint64_t da0 = sdesc(su32(sh.a[0][0]), 128, (BK / 8) * 128);
      const uint64_t db0 = sdesc(su32(sh.b[0][0]), 128, (BK / 8) * 128);
      for (int p = 0; p < 2 && ok; ++p) {
        int lo, hi;
        kb_range(p, g, i0, j0, lo, hi);
        int since = 0;  // K blocks of the current chunk of the leading weights
        for (int kb = lo; kb < hi; ++kb) {
          if (!mbar_wait(&sh.full[st], ph, err, timeout_ns)) {
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
          const uint64_t da = da0 + st * kDescStageA, db = db0 + st * kDescStageB;
          // weights above kLeadW first (their accumulators live for the whole product),
          // then the leading ones, once their previous chunk has been drained
          issue_part<false, MAXW, SMAX>(tbase, da, db, kb != lo ? 1u : 0u);
          if (pend >= 0) {
            if (!mbar_wait(&sh.accempty, pend & 1, err, timeout_ns)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            pend = -1;
          }
          issue_part<true, MAXW, SMAX>(tbase, da, db, since != 0 ? 1u : 0u);
          umma_commit(&sh.empty[st]);
          if (++st == NST) {
            st = 0;
            ph ^= 1;
          }
          ++since;
          const bool last = kb == hi - 1;
          if (last || since == kLeadStages) {
            umma_commit(&sh.accfull);
            pend = ev++;
            pend_all = last;
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
    // R is written once per product: the first product's drain writes R = C - P_0, a
    // later one R -= P_1; mx is the largest |R| written by the last pass.  Each pass
    // reads its values in chunks of 8 before storing any (the compiler cannot move a
    // load above a store that may alias it, so element by element every access would
    // be a memory round trip of its own).
    bool wrote = false;
    double mx = 0.0;
    // Leading weights of each column, over the chunks of a product:
    //   L = 2^16 S_2 + 2^8 S_3 + S_4   (S_w the integer sum of weight w),
    // so that their part of the product is 2^(e_row + e_col - 32) L.  A chunk adds
    // less than 2^24 (2^16 + 2^8 + 1) < 2^40.01 in magnitude, so L is exact in int64
    // for up to 2^22 chunks (K below 8 * 10^8) and exact in binary64 below 2^12
    // chunks (K below 786432); beyond that its conversion rounds once, by 2^-53.
    long long lacc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) lacc[j] = 0;
    int ev = 0;
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
      int lo, hi;
      kb_range(p, g, i0, j0, lo, hi);
      if (hi <= lo) continue;  // no second product (dense form): nothing committed, nothing to drain
      const int erow = g.a[p].e[gi];
      const int nst = hi - lo;
      const int nlead = (nst - 1) / kLeadStages;  // drains of the leading weights before the last
      for (int d = 0; d <= nlead && ok; ++d, ++ev) {
        const bool last = d == nlead;  // the same in every lane (TMEM loads are warp-collective)
        if (!mbar_wait(&sh.accfull, ev & 1, err, timeout_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t v2[16], v3[16], v4[16];
          tmem_ld16(tl + static_cast<uint32_t>(0 * BN + cb0 + 16 * h), v2);
          tmem_ld16(tl + static_cast<uint32_t>(1 * BN + cb0 + 16 * h), v3);
          tmem_ld16(tl + static_cast<uint32_t>(2 * BN + cb0 + 16 * h), v4);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {  // the integer sums S_2, S_3, S_4 (exact)
            const long long c2 = __float2int_rn(__uint_as_float(v2[j]));
            const long long c3 = __float2int_rn(__uint_as_float(v3[j]) * 0x1p8f);
            const int c4 = __float2int_rn(__uint_as_float(v4[j]) * 0x1p16f);
            lacc[16 * h + j] += c2 * 65536 + c3 * 256 + c4;
          }
        }
        // The accumulators of the weights w >= 5 hold 2^(-8(w-2)) S_w; their sum T'
        // is formed in binary32 from the smallest weight up (one more rounding of
        // 2^-24 T', the size of the accumulation's own), and the product is
        // 2^(e_row + e_col - 32) (L + 2^16 T').  Everything leaves TMEM before the
        // accumulators are handed back, so the binary64 update below overlaps the
        // next product's MMAs.
        float tf[32];
        if (last) {
#pragma unroll
          for (int j = 0; j < 32; ++j) tf[j] = 0.0f;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int w = MAXW; w > kLeadW; --w) {
              uint32_t v[16];
              tmem_ld16(tl + static_cast<uint32_t>((w - 2) * BN + cb0 + 16 * h), v);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 16; ++j) tf[16 * h + j] += __uint_as_float(v[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh.accempty);
        if (last) {
          // R = (C, or R after an earlier product) - 2^(e_row + e_col - 32) (L + 2^16 T')
          const double* src = wrote ? R : C;
          const int64_t lds = wrote ? ldr : ldc;
          mx = 0.0;
          if (gi < m)
#pragma unroll
            for (int c8 = 0; c8 < 32; c8 += 8) {
              double v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int64_t gj = j0 + cb0 + c8 + j;
                v[j] = gj < n ? src[gi + gj * lds] : 0.0;
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int64_t gj = j0 + cb0 + c8 + j;
                if (gj < n) {
                  const long long L = lacc[c8 + j];
                  double r = v[j];
                  if (L != 0 || tf[c8 + j] != 0.0f) {
                    const double dv = fma(static_cast<double>(tf[c8 + j]), 0x1p16, static_cast<double>(L));
                    r -= mul2(dv, erow + sh.ecol[p][cb0 + c8 + j] - 32);
                  }
                  R[gi + gj * ldr] = r;
                  mx = fmax(mx, fabs(r));
                }
              }
            }
          wrote = true;
#pragma unroll
          for (int j = 0; j < 32; ++j) lacc[j] = 0;
        }
      }
    }
    if (ok && !wrote && gi < m)  // no product drained (no K blocks): R = C
      for (int j = 0; j < 32; ++j) {
        const int64_t gj = j0 + cb0 + j;
        if (gj < n) {
          const double r = C[gi + gj * ldc];
          R[gi + gj * ldr] = r;
          mx = fmax(mx, fabs(r));
        }
      }
    if (!ok) atomicCAS(err, 0, SYLV_ERR_TIMEOUT);
    // ---- max |R| of the tile (from the last pass)
    mx = warp_max(mx);
    if (lane == 0 && rmax && !ld_volatile(err)) atomic_max_nonneg(rmax, mx);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

template <int MAXW>
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_gemm(Gemm g, const double* C, int64_t ldc, double* R, int64_t ldr, int64_t m, int64_t n,
              unsigned long long* rmax, int* err, long long timeout_ns, const int* skip) {
  if (skip && ld_volatile(skip)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& sh = *reinterpret_cast<Smem*>(smem_raw);
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
  oz_tile<MAXW>(sh, g, C, ldc, R, ldr, m, n, rmax, err, timeout_ns, mb, nb);
}

// ---- batched residuals: many independent equations, one launch per step.
// Packed operand shapes of an m x n equation (see the host's carving): operand 0 is
// A (rows of A, K = its columns), 1 X by columns, 2 X by rows, 3 B by columns.
__host__ __device__ inline void oz_shape(int64_t m, int64_t n, int which, int64_t& RB, int64_t& KB, int& R) {
  const int64_t rows = (which == 0 || which == 2) ? m : n;
  const int64_t kd = (which <= 1) ? m : n;
  R = (which == 0 || which == 2) ? BM : BN;
  RB = (rows + R - 1) / R;
  KB = (kd + BK - 1) / BK;
}
__device__ __forceinline__ Packed oz_packed(const OzBatchEq& q, int which) {
  Packed P;
  P.p = static_cast<__nv_bfloat16*>(q.b.p[which]);
  P.e = q.b.e[which];
  oz_shape(q.b.m, q.b.n, which, P.RB, P.KB, P.R);
  return P;
}
__device__ __forceinline__ View oz_view(const OzBatchEq& q, int which) {
  const int64_t m = q.b.m, n = q.b.n;
  switch (which) {
    case 0: return View{q.A, 1, q.lda, m, m, 1};   // A as rows, r <= k + 1
    case 1: return View{q.X, q.ldx, 1, n, m, 0};   // X by columns: element (j, i) = X[i, j]
    case 2: return View{q.X, 1, q.ldx, m, n, 0};   // X by rows
    default: return View{q.B, q.ldb, 1, n, n, 2};  // B by columns: element (j, k) = B[k, j], k <= j + 1
  }
}

// Per-row exponents of operand `which` of every equation (equation blockIdx.y).
__global__ void k_oz_rowexp_batched(const OzBatchEq* __restrict__ eqs, int which) {
  const OzBatchEq& q = eqs[blockIdx.y];
  if (!q.active || (q.skip && ld_volatile(q.skip))) return;
  const Packed P = oz_packed(q, which);
  oz_rowexp(oz_view(q, which), P.e, P.RB * P.R);
}

// Slices of operand `which` of every equation (equation blockIdx.y).
__global__ void __launch_bounds__(256) k_oz_split_batched(const OzBatchEq* __restrict__ eqs, int which) {
  __shared__ double tile[BM * (BK + 1)];
  const OzBatchEq& q = eqs[blockIdx.y];
  if (!q.active || (q.skip && ld_volatile(q.skip))) return;
  oz_split(oz_view(q, which), oz_packed(q, which), tile);
}

// One output tile per CTA from the task list (equation, row panel, column panel).
template <int MAXW>
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_gemm_batched(const OzBatchEq* __restrict__ eqs, const OzTask* __restrict__ tasks, int* err,
                      long long timeout_ns) {
  const OzTask t = tasks[blockIdx.x];
  const OzBatchEq& q = eqs[t.eq];
  if (q.skip && ld_volatile(q.skip)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& sh = *reinterpret_cast<Smem*>(smem_raw);
  // The equation's operand descriptors in shared memory (registers are scarce in the
  // drain warps).
  if (threadIdx.x < 4) {
    const Packed P = oz_packed(q, threadIdx.x);
    if (threadIdx.x & 1)
      sh.g.b[threadIdx.x >> 1] = P;
    else
      sh.g.a[threadIdx.x >> 1] = P;
  }
  if (threadIdx.x == 0) sh.g.dense = 0;
  __syncthreads();
  oz_tile<MAXW>(sh, sh.g, q.C, q.ldc, q.R, q.ldr, q.b.m, q.b.n, q.rmax, err, timeout_ns, t.mb, t.nb);
}

}  // namespace oz
}  // namespace sylv
