// sylv_prep.cuh -- kernels around the tile DAG: structure scan and tile
// partition, tile norms, the level-ordered task list, consistency scaling,
// per-equation results, and the index reversals that reduce transposed problems
// to the untransposed one.
#pragma once

#include "sylv_internal.cuh"

namespace sylv {

// ---------------------------------------------------------------------------
// Structure scan and tile partition (Sec. 1 eq. (4); Sec. 2.2).  One CTA per
// (equation, matrix): marks every i with M[i+1,i] != 0 (a 2x2 block at i), rejects
// two consecutive marks, then places tile boundaries greedily: the next boundary
// is b + t, moved back to b + t - 1 when that would split a 2x2 block.  Tiles are
// therefore t or t-1 rows (the last may be shorter) and diagonal tiles are square.
template <typename T>
__global__ void k_scan(Work w) {
  extern __shared__ unsigned int bits[];
  const Inst I = w.inst[blockIdx.x];
  InstState* st = &w.st[blockIdx.x];
  const bool isA = blockIdx.y == 0;
  const int64_t N = isA ? I.m : I.n;
  const int64_t ld = isA ? I.lda : I.ldb;
  const T* M = static_cast<const T*>(isA ? I.A : I.B);
  const bool scan = isA || !I.nob;  // without a B term the columns of C are partitioned freely
  const int64_t nwords = (N + 31) / 32;
  for (int64_t i = threadIdx.x; i < nwords; i += blockDim.x) bits[i] = 0u;
  __syncthreads();
  if (scan)
    for (int64_t i = threadIdx.x; i + 1 < N; i += blockDim.x)
      if (M[(i + 1) + i * ld] != T(0)) atomicOr(&bits[i >> 5], 1u << (i & 31));
  __syncthreads();
  for (int64_t wd = threadIdx.x; wd < nwords; wd += blockDim.x) {
    const unsigned x = bits[wd];
    const unsigned nxt = (wd + 1 < nwords) ? bits[wd + 1] : 0u;
    if ((x & (x >> 1)) || ((x >> 31) & nxt & 1u)) set_err(st, isA ? SYLV_ERR_STRUCTURE_A : SYLV_ERR_STRUCTURE_B);
  }
  if (threadIdx.x == 0) {
    int32_t* bnd = w.ibuf + (isA ? I.rb : I.cb);
    const int cap = isA ? I.pmax : I.qmax;
    int64_t b = 0;
    int cnt = 0;
    bnd[0] = 0;
    while (b < N) {
      int64_t e = b + I.t < N ? b + I.t : N;
      if (e < N && ((bits[(e - 1) >> 5] >> ((e - 1) & 31)) & 1u)) e -= 1;
      if (cnt >= cap) {
        set_err(st, SYLV_ERR_WORKSPACE);
        break;
      }
      bnd[++cnt] = static_cast<int32_t>(e);
      b = e;
    }
    if (isA)
      st->p = cnt;
    else
      st->q = cnt;
  }
}

// ---------------------------------------------------------------------------
// Bound (Sec. 2.2): infinity norms of the tiles of A (row tile i, column tile
// k >= i) and of B, computed once before the DAG starts, plus max |entry|
// (for the pivot floor), NaN/Inf detection and the ||tile|| <= Omega
// precondition.  grid = (equation, row tile, matrix); a warp per column tile.
template <typename T>
__global__ void k_norms(Work w) {
  const Inst I = w.inst[blockIdx.x];
  InstState* st = &w.st[blockIdx.x];
  const bool isA = blockIdx.z == 0;
  if (!isA && I.nob) return;
  const int ntile = isA ? st->p : st->q;
  const int rt = blockIdx.y;
  if (rt >= ntile || st->err) return;
  const int64_t ld = isA ? I.lda : I.ldb;
  const T* M = static_cast<const T*>(isA ? I.A : I.B);
  const int32_t* bnd = w.ibuf + (isA ? I.rb : I.cb);
  double* out = w.dbuf + (isA ? I.an : I.bn);
  const int cap = isA ? I.pmax : I.qmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int rs = bnd[rt], re = bnd[rt + 1];
  // Per element only the sum's addition is floating point: the maximum and the finite
  // test work on the bit patterns (a binary64 instruction costs 64 binary32 ones).  A
  // binary32 tile sums in binary32 rounded upwards (an upper bound of its norm).
  constexpr bool kF32 = sizeof(T) == 4;
  using Bits = typename std::conditional<kF32, unsigned, unsigned long long>::type;
  constexpr Bits kMag = kF32 ? Bits(0x7fffffffu) : Bits(0x7FFFFFFFFFFFFFFFull);
  constexpr Bits kInf = kF32 ? Bits(0x7f800000u) : Bits(0x7FF0000000000000ull);
  Bits emax = 0;
  bool bad = false;
  for (int ct = rt + warp; ct < ntile; ct += nwarp) {
    const int cs = bnd[ct], ce = bnd[ct + 1];
    double best = 0.0;
    for (int r = rs + lane; r < re; r += 32) {
      T s = T(0);
      for (int c = cs; c < ce; ++c) {
        if (r > c + 1) continue;
        Bits b;
        memcpy(&b, &M[r + static_cast<int64_t>(c) * ld], sizeof(T));
        b &= kMag;
        if (b >= kInf) bad = true;
        emax = b > emax ? b : emax;
        T v;
        memcpy(&v, &b, sizeof(T));
        if constexpr (kF32)
          s = __fadd_ru(s, v);
        else
          s += v;
      }
      best = fmax(best, static_cast<double>(s));
    }
    best = warp_max(best);
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      out[static_cast<int64_t>(rt) * cap + ct] = best;
      if (any_bad)
        set_err(st, SYLV_ERR_NONFINITE);
      else if (best > I.omega)
        set_err(st, SYLV_ERR_RANGE);
    }
  }
  if (bad) set_err(st, SYLV_ERR_NONFINITE);
  for (int o = 16; o > 0; o >>= 1) {
    const Bits u = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = u > emax ? u : emax;
  }
  if (lane == 0 && emax && emax < kInf) {
    T v;
    memcpy(&v, &emax, sizeof(T));
    atomic_max_nonneg(isA ? &st->amax : &st->bmax, static_cast<double>(v));
  }
}

// ---------------------------------------------------------------------------
// Task list: every tile (k,l) of every valid equation, ordered by its
// anti-diagonal level d = (p-1-k) + l (all producers of a tile sit on lower
// levels, so ticket order is a topological order).  Also sets the pivot floor
// smin = max(2^-52 max(|A|,|B|), 2^-1022).
__global__ void k_level_count(Work w) {
  const int lw = w.inst[blockIdx.x].nob ? 0 : 1;  // without a B term a tile waits only on the tiles below it
  InstState* st = &w.st[blockIdx.x];
  if (threadIdx.x == 0) {
    const double amax = __longlong_as_double(static_cast<long long>(st->amax));
    const double bmax = __longlong_as_double(static_cast<long long>(st->bmax));
    st->smin = fmax(0x1p-52 * fmax(amax, bmax), 0x1p-1022);
  }
  if (st->err) return;
  const int p = st->p, q = st->q;
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) {
    const int k = t / q, l = t % q;
    atomicAdd(&w.lvl_cnt[(p - 1 - k) + lw * l], 1);
  }
}

__global__ void k_level_scan(Work w) {
  if (threadIdx.x == 0) {
    int run = 0, used = 0;
    for (int d = 0; d < w.nlevels_max; ++d) {
      w.lvl_off[d] = run;
      run += w.lvl_cnt[d];
      if (w.lvl_cnt[d]) used = d + 1;
    }
    w.ctrl->ntasks = run;
    w.ctrl->nlevels = used;
  }
}

__global__ void k_level_scatter(Work w) {
  const Inst I = w.inst[blockIdx.x];
  InstState* st = &w.st[blockIdx.x];
  if (st->err) return;
  const int p = st->p, q = st->q;
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) {
    const int k = t / q, l = t % q;
    const int d = (p - 1 - k) + (I.nob ? 0 : l);
    const int pos = atomicAdd(&w.lvl_cur[d], 1);
    w.tasks[w.lvl_off[d] + pos] = Task{static_cast<int32_t>(blockIdx.x), k * I.qmax + l};
  }
}

// ---------------------------------------------------------------------------
// Consistency scaling (end of Algorithm 4): alpha = min_kl alpha_kl, and every
// tile with a larger local factor is multiplied by alpha / alpha_kl = 2^(E - e_kl).
// Packed operand tiles (see Work::pack): A_ki for i > k in the left-operand layout
// (L[kk * LDG + r] = A[row r of tile k, column kk of tile i]) and B_jl for j < l in
// the right-operand layout (R[kk * LDG + c] = B[row kk of tile j, column c of tile
// l]), zero outside the tiles, LDG = tt + 2.  Grid (equations, blocks per
// equation); B tiles go through shared memory so that reads and writes coalesce.
template <typename T>
__global__ void __launch_bounds__(256) k_pack(Work w, int tt) {
  __shared__ T tb[64 * 65];
  const Inst I = w.inst[blockIdx.x];
  const int p = w.st[blockIdx.x].p, q = w.st[blockIdx.x].q;
  const int32_t* rb = w.ibuf + I.rb;
  const int32_t* cb = w.ibuf + I.cb;
  const int LDG = tt + 2, nel = tt * LDG;
  const T* A = static_cast<const T*>(I.A);
  const T* B = static_cast<const T*>(I.B);
  const int64_t na = static_cast<int64_t>(p) * p, nb = static_cast<int64_t>(q) * q;
  for (int64_t sidx = blockIdx.y; sidx < na + nb; sidx += gridDim.y) {
    if (sidx < na) {
      const int k = static_cast<int>(sidx / p), i = static_cast<int>(sidx % p);
      if (i <= k) continue;
      const int r0 = rb[k], mt = rb[k + 1] - r0, k0 = rb[i], kd = rb[i + 1] - k0;
      T* dst = reinterpret_cast<T*>(w.pack + pack_a(I, k, i) * w.pack_slot);
      for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
        const int kk = idx / LDG, r = idx % LDG;
        dst[idx] = (r < mt && kk < kd) ? A[(r0 + r) + static_cast<int64_t>(k0 + kk) * I.lda] : T(0);
      }
    } else {
      if (I.nob) break;  // no B term
      const int64_t s2 = sidx - na;
      const int j = static_cast<int>(s2 / q), l = static_cast<int>(s2 % q);
      if (l <= j) continue;
      const int k0 = cb[j], kd = cb[j + 1] - k0, c0 = cb[l], nt = cb[l + 1] - c0;
      __syncthreads();  // the previous tile's reads of tb are done
      for (int idx = threadIdx.x; idx < tt * tt; idx += blockDim.x) {
        const int kk = idx % tt, c = idx / tt;
        tb[c * (tt + 1) + kk] = (kk < kd && c < nt) ? B[(k0 + kk) + static_cast<int64_t>(c0 + c) * I.ldb] : T(0);
      }
      __syncthreads();
      T* dst = reinterpret_cast<T*>(w.pack + pack_b(I, j, l) * w.pack_slot);
      for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
        const int kk = idx / LDG, c = idx % LDG;
        dst[idx] = (c < tt) ? tb[c * (tt + 1) + kk] : T(0);
      }
    }
  }
}

template <typename T>
__global__ void k_consistency(Work w) {
  const int ntasks = w.ctrl->ntasks;
  for (int idx = blockIdx.x; idx < ntasks; idx += gridDim.x) {
    const Task tk = w.tasks[idx];
    const Inst I = w.inst[tk.inst];
    if (!I.robust) continue;
    const InstState* st = &w.st[tk.inst];
    const int E = st->minexp;
    const int e = w.texp[I.tile + tk.tile];
    if (e == E) continue;
    const int k = tk.tile / I.qmax, l = tk.tile % I.qmax;
    const int32_t* rb = w.ibuf + I.rb;
    const int32_t* cb = w.ibuf + I.cb;
    const int r0 = rb[k], mt = rb[k + 1] - r0, c0 = cb[l], nt = cb[l + 1] - c0;
    T* C = static_cast<T*>(I.C);
    for (int i = threadIdx.x; i < mt * nt; i += blockDim.x) {
      T* p = &C[(r0 + i % mt) + static_cast<int64_t>(c0 + i / mt) * I.ldc];
      *p = mul2(*p, E - e);
    }
  }
}

// Per-equation result record (status precedence: launch error, input error,
// overflow in non-robust mode, double underflow of alpha, near singularity).
__global__ void k_results(Work w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.count; i += gridDim.x * blockDim.x) {
    const Inst I = w.inst[i];
    const InstState* st = &w.st[i];
    sylv_result r;
    const int E = I.robust ? st->minexp : 0;
    r.log2scale = E;
    r.scale = mul2(1.0, E);
    int info = SYLV_OK;
    if (w.ctrl->err)
      info = w.ctrl->err;
    else if (st->err)
      info = st->err;
    else if (st->flags & kFlagNonfiniteOut)
      info = SYLV_OVERFLOWED;
    else if (r.scale == 0.0)
      info = SYLV_SCALE_UNDERFLOW;
    else if (st->flags & kFlagNearSingular)
      info = SYLV_NEAR_SINGULAR;
    r.info = info;
    r.iters = 0;
    r.last_update = 0.0;
    r.scale_events = st->nscale;
    r.min_tile_exp = st->minexp;
    w.res[i] = r;
  }
}

// ---------------------------------------------------------------------------
// Transposes: op(A)^T problems become untransposed ones by reversing indices,
// A^T Y + Y B = C  <=>  (J A^T J)(J Y) + (J Y) B = J C,  J the reversal permutation;
// J A^T J is upper quasi-triangular when A is.  dst = J src^T J restricted to the
// quasi-triangular part (other entries 0), through a 32x32 shared-memory tile.
// dst(i, j) = sign * src(N-1-j, N-1-i) on the quasi-triangular part; one block
// covers dst rows i0.., cols j0.. (32 x 8 threads).
template <typename T>
__device__ __forceinline__ void k_anti_transpose_body(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                                      int64_t ldd, int64_t N, T sign, T (&tile)[32][33], int64_t i0,
                                                      int64_t j0, int tx, int ty) {
  // source rows N-1-j (j in j0..j0+31), source cols N-1-i (i in i0..i0+31)
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = i0 + yy, j = j0 + tx;  // read coalesced along source rows = N-1-j
    T v = T(0);
    if (i < N && j < N) v = src[(N - 1 - j) + (N - 1 - i) * lds];
    tile[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t j = j0 + yy, i = i0 + tx;
    if (i < N && j < N) dst[i + j * ldd] = (i <= j + 1) ? sign * tile[tx][yy] : T(0);
  }
}
template <typename T>
__global__ void k_anti_transpose(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd,
                                 int64_t N) {
  __shared__ T tile[32][33];
  k_anti_transpose_body(src, lds, dst, ldd, N, T(1), tile, static_cast<int64_t>(blockIdx.x) * 32,
                        static_cast<int64_t>(blockIdx.y) * 32, static_cast<int>(threadIdx.x & 31),
                        static_cast<int>(threadIdx.x >> 5));
}

// dst = sign * op(src) on the quasi-triangular part: op = J src^T J (trans) or the
// identity.  The anti-transpose turns op(B) = B^T into an upper quasi-triangular
// matrix; the sign turns A Y - Y B into A Y + Y (-B).
template <typename T>
__global__ void k_operand_copy(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd, int64_t N,
                               int trans, T sign) {
  __shared__ T tile[32][33];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * 32, j0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (trans) {
    k_anti_transpose_body(src, lds, dst, ldd, N, sign, tile, i0, j0, tx, ty);
    return;
  }
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = i0 + tx, j = j0 + yy;
    if (i < N && j < N) dst[i + j * ldd] = (i <= j + 1) ? sign * src[i + j * lds] : T(0);
  }
}

// In-place reversal of the rows (dim = 0) or columns (dim = 1) of an m x n matrix.
template <typename T>
__global__ void k_flip(T* C, int64_t ldc, int64_t m, int64_t n, int dim) {
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
    T a = C[i + j * ldc], b = C[i2 + j2 * ldc];
    C[i + j * ldc] = b;
    C[i2 + j2 * ldc] = a;
  }
}

}  // namespace sylv

namespace sylv {

// ---------------------------------------------------------------------------
// Batched forms of the transposition helpers (one launch for all equations).
struct TransDesc {
  const double* src;
  int64_t lds;
  double* dst;  // N x N, leading dimension N
  int64_t N;
  int32_t trans;  // anti-transpose (op = ^T) or plain copy
  int32_t pad;
  double sign;    // -1 for the B operand of isgn = -1
};

// dst_e = sign_e * op(src_e) (quasi-triangular part; op = J .^T J or the identity) for every
// equation e = blockIdx.z.
__global__ void k_anti_transpose_batched(const TransDesc* __restrict__ d) {
  __shared__ double tile[32][33];
  const TransDesc D = d[blockIdx.z];
  const int64_t N = D.N;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * 32, j0 = static_cast<int64_t>(blockIdx.y) * 32;
  if (i0 >= N || j0 >= N) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (D.trans) {
    k_anti_transpose_body(D.src, D.lds, D.dst, N, N, D.sign, tile, i0, j0, tx, ty);
    return;
  }
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = i0 + tx, j = j0 + yy;
    if (i < N && j < N) D.dst[i + j * N] = (i <= j + 1) ? D.sign * D.src[i + j * D.lds] : 0.0;
  }
}

// In-place reversal of the rows (dim 0) or columns (dim 1) of every equation's C
// (equation e = blockIdx.y).
__global__ void k_flip_batched(const Inst* __restrict__ inst, int dim) {
  const Inst I = inst[blockIdx.y];
  double* C = static_cast<double*>(I.C);
  const int64_t m = I.m, n = I.n;
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
    const double a = C[i + j * I.ldc], b = C[i2 + j2 * I.ldc];
    C[i + j * I.ldc] = b;
    C[i2 + j2 * I.ldc] = a;
  }
}

}  // namespace sylv
