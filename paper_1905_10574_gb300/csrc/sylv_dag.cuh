// sylv_dag.cuh -- the persistent tile-DAG kernel of the robust tiled solver
// (Algorithm 4 of Schwarz & Kjelgaard Mikkelsen 2019), templated on the tile
// capacity TT, the element type T and robust/non-robust mode.
//
// Work decomposition.  Tile (k,l) of Y (0-based, p x q tiles) depends on tiles
// (i,l), i > k, through Y_kl -= A_ki Y_il and on tiles (k,j), j < l, through
// Y_kl -= Y_kj B_jl (the block form of eq. (6)/(7), with the index ranges that an
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

#include "sylv_internal.cuh"

namespace sylv {

template <int TT, typename T>
struct DagSmem {
  static constexpr int LDG = TT + 2;  // row stride of the GEMM operands (16-byte aligned rows)
  static constexpr int LDY = TT + 1;  // leading dimension of the Y, A_kk, B_ll tiles
  T L[TT * LDG];                      // left GEMM operand, k-major; A_kk in the diagonal phase
  T R[TT * LDG];                      // right GEMM operand, k-major; B_ll in the diagonal phase
  T Y[TT * LDY];                      // the tile being solved (column-major)
  double zbuf[TT][4];                 // this step's solved 1x1/2x2 blocks, by block column
  double acolmax[TT];                 // per A block: max row-sum of A above it (within the tile)
  double browmax[TT];                 // per B block: max block norm of B right of it
  double pzn[TT];                     // norm of each solved block of this step
  int pe[TT];                         // scale exponent of each solved block of this step
  short rowblk[TT], colblk[TT];       // block index of every row / column of the tile
  short astart[TT + 1], bstart[TT + 1];
  unsigned long long umax;
  double nb_acc, U;
  int task, abort, e_acc, sacc, sop, g, e_diag, pb, qb, nscale, flags;
};

// ----------------------------------------------------------------------------
// Robust solve of a small Sylvester system A11 Z + Z B11 = beta R with A11 ma x ma,
// B11 nb x nb (ma, nb in {1,2}) through its (ma nb)-square Kronecker system
// (I (x) A11 + B11^T (x) I) vec Z = beta vec R, by Gaussian elimination with complete
// pivoting (Sec. 2.1).  Right-hand-side updates are guarded by ProtectUpdate and
// divisions by ProtectDivision; the guards' exponents add up to log2(beta), which
// is returned.  Pivots below smin are raised to smin (*near = true).  a and b are
// the blocks column-major (ld 2); r is R column-major (ld ma) on entry, Z on exit.
__device__ inline int small_sylv(int ma, int nb, const double* a, const double* b, double* r,
                                 double smin, double omega, bool robust, bool* near) {
  const int s = ma * nb;
  double M[4][4];
  int cp[4];
  int lb = 0;
  for (int u = 0; u < s; ++u) {
    const int i = u % ma, j = u / ma;
    cp[u] = u;
    for (int v = 0; v < s; ++v) {
      const int i2 = v % ma, j2 = v / ma;
      double e = 0.0;
      if (j == j2) e += a[i + 2 * i2];
      if (i == i2) e += b[j2 + 2 * j];
      M[u][v] = e;
    }
  }
  for (int st = 0; st < s; ++st) {
    int pr = st, pc = st;
    double best = -1.0;
    for (int u = st; u < s; ++u)
      for (int v = st; v < s; ++v) {
        const double mag = fabs(M[u][v]);
        if (mag > best) {
          best = mag;
          pr = u;
          pc = v;
        }
      }
    if (pr != st) {
      for (int v = 0; v < s; ++v) {
        const double tmp = M[st][v];
        M[st][v] = M[pr][v];
        M[pr][v] = tmp;
      }
      const double tmp = r[st];
      r[st] = r[pr];
      r[pr] = tmp;
    }
    if (pc != st) {
      for (int u = 0; u < s; ++u) {
        const double tmp = M[u][st];
        M[u][st] = M[u][pc];
        M[u][pc] = tmp;
      }
      const int tmp = cp[st];
      cp[st] = cp[pc];
      cp[pc] = tmp;
    }
    if (fabs(M[st][st]) < smin) {
      M[st][st] = smin;
      *near = true;
    }
    for (int u = st + 1; u < s; ++u) {
      const double l = M[u][st] / M[st][st];
      for (int v = st + 1; v < s; ++v) M[u][v] = fma(-l, M[st][v], M[u][v]);
      if (robust) {
        const int z = protect_update(fabs(r[u]), fabs(l), fabs(r[st]), omega);
        if (z) {
          for (int w = 0; w < s; ++w) r[w] = mul2(r[w], z);
          lb += z;
        }
      }
      r[u] = fma(-l, r[st], r[u]);
    }
  }
  for (int i = s - 1; i >= 0; --i) {
    for (int v = i + 1; v < s; ++v) {
      if (robust) {
        const int z = protect_update(fabs(r[i]), fabs(M[i][v]), fabs(r[v]), omega);
        if (z) {
          for (int w = 0; w < s; ++w) r[w] = mul2(r[w], z);
          lb += z;
        }
      }
      r[i] = fma(-M[i][v], r[v], r[i]);
    }
    if (robust) {
      const int z = protect_division(r[i], M[i][i], omega);
      if (z) {
        for (int w = 0; w < s; ++w) r[w] = mul2(r[w], z);
        lb += z;
      }
    }
    r[i] = r[i] / M[i][i];
  }
  double x[4];
  for (int u = 0; u < s; ++u) x[cp[u]] = r[u];
  for (int u = 0; u < s; ++u) r[u] = x[u];
  return lb;
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

// Diagonal-tile solve: Algorithm 2 applied to one tile, in wavefront order.
// Small blocks (kb, lb) on the anti-diagonal s = (pb-1-kb) + lb are independent;
// each step solves them (one thread per block), agrees on one tile-wide scale
// factor, and pushes their contributions to the unsolved elements (each element is
// updated by the thread that owns it, so no two threads write one element).
// Robustness: U bounds the block norms of every unsolved block; per step
//   g = e_min + ProtectUpdate twice, so that 2^g (U + As*Zs + Zs*Bs) <= omega,
// where Zs bounds the step's solved block norms, As the norms of the A blocks
// above them and Bs the norms of the B blocks right of them.  Every element of the
// tile is multiplied by 2^g (exactly), the step's blocks by 2^(g - e_block).
template <int TT, typename T, bool ROBUST>
__device__ void diag_solve(DagSmem<TT, T>& sh, int mt, int nt, double omega, double smin) {
  constexpr int LDY = DagSmem<TT, T>::LDY;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* Ak = sh.L;
  const T* Bk = sh.R;
  T* Ys = sh.Y;

  if (warp == 0) {
    const int pb = scan_blocks<T, LDY>(Ak, mt, sh.rowblk, sh.astart, lane);
    if (lane == 0) sh.pb = pb;
  } else if (warp == 1) {
    const int qb = scan_blocks<T, LDY>(Bk, nt, sh.colblk, sh.bstart, lane);
    if (lane == 0) sh.qb = qb;
  }
  if (tid == 0) {
    sh.umax = 0ull;
    sh.e_diag = 0;
  }
  __syncthreads();
  const int pb = sh.pb, qb = sh.qb;

  if (ROBUST) {
    for (int kb = tid; kb < pb; kb += kThreads) {
      const int ra = sh.astart[kb], re = sh.astart[kb + 1];
      double best = 0.0;
      for (int r = 0; r < ra; ++r) {
        double s = 0.0;
        for (int i = ra; i < re; ++i) s += fabs(static_cast<double>(Ak[r + i * LDY]));
        best = fmax(best, s);
      }
      sh.acolmax[kb] = best;
    }
    for (int lb = tid; lb < qb; lb += kThreads) {
      const int c0 = sh.bstart[lb], c1 = sh.bstart[lb + 1];
      double best = 0.0;
      for (int jb = lb + 1; jb < qb; ++jb) {
        const int j0 = sh.bstart[jb], j1 = sh.bstart[jb + 1];
        for (int row = c0; row < c1; ++row) {
          double s = 0.0;
          for (int c = j0; c < j1; ++c) s += fabs(static_cast<double>(Bk[row + c * LDY]));
          best = fmax(best, s);
        }
      }
      sh.browmax[lb] = best;
    }
    // U0: largest block infinity norm of the tile.
    for (int idx = tid; idx < mt * nt; idx += kThreads) {
      const int r = idx % mt, c = idx / mt;
      const int lbc = sh.colblk[c];
      if (sh.bstart[lbc] != c) continue;
      double s = fabs(static_cast<double>(Ys[r + c * LDY]));
      if (sh.bstart[lbc + 1] - c == 2) s += fabs(static_cast<double>(Ys[r + (c + 1) * LDY]));
      atomic_max_nonneg(&sh.umax, s);
    }
  }
  __syncthreads();
  if (tid == 0) sh.U = __longlong_as_double(static_cast<long long>(sh.umax));

  // Element ownership in the update phase: thread owns row tid % TT, columns
  // tid / TT + j * (kThreads / TT).
  constexpr int CSTEP = kThreads / TT;
  const int my_r = tid % TT;
  const int my_c0 = tid / TT;
  const bool row_ok = my_r < mt;
  const int kb_r = row_ok ? sh.rowblk[my_r] : 0;
  const int dr = pb - 1 - kb_r;
  const int ra_r = row_ok ? sh.astart[kb_r] : 0;
  const int ma_r = row_ok ? sh.astart[kb_r + 1] - ra_r : 1;
  bool near = false;
  int local_scale_events = 0;

  const int nsteps = pb + qb - 1;
  for (int s = 0; s < nsteps; ++s) {
    const int lb_lo = max(0, s - (pb - 1));
    const int lb_hi = min(s, qb - 1);
    // Phase A: solve this step's blocks.
    for (int lb = lb_lo + tid; lb <= lb_hi; lb += kThreads) {
      const int kb = pb - 1 - (s - lb);
      const int r0 = sh.astart[kb], ma = sh.astart[kb + 1] - r0;
      const int c0 = sh.bstart[lb], nb = sh.bstart[lb + 1] - c0;
      double a[4], b[4], rr[4];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          a[i + 2 * j] = (i < ma && j < ma) ? static_cast<double>(Ak[(r0 + i) + (r0 + j) * LDY]) : 0.0;
          b[i + 2 * j] = (i < nb && j < nb) ? static_cast<double>(Bk[(c0 + i) + (c0 + j) * LDY]) : 0.0;
        }
      for (int u = 0; u < ma * nb; ++u)
        rr[u] = static_cast<double>(Ys[(r0 + u % ma) + (c0 + u / ma) * LDY]);
      const int e = small_sylv(ma, nb, a, b, rr, smin, omega, ROBUST, &near);
      double zn = 0.0;
      for (int i = 0; i < ma; ++i) {
        double rs = 0.0;
        for (int j = 0; j < nb; ++j) rs += fabs(rr[i + ma * j]);
        zn = fmax(zn, rs);
      }
      for (int u = 0; u < 4; ++u) sh.zbuf[lb][u] = (u < ma * nb) ? rr[u] : 0.0;
      sh.pe[lb] = e;
      sh.pzn[lb] = zn;
    }
    __syncthreads();
    // Phase B: one tile-wide scale factor for this step.
    if (ROBUST) {
      if (warp == 0) {
        int emin = 0;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) emin = min(emin, sh.pe[lb]);
        emin = warp_min(emin);
        double zs = 0.0, as = 0.0, bs = 0.0;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) {
          const int kb = pb - 1 - (s - lb);
          zs = fmax(zs, mul2(sh.pzn[lb], emin - sh.pe[lb]));
          as = fmax(as, sh.acolmax[kb]);
          bs = fmax(bs, sh.browmax[lb]);
        }
        zs = warp_max(zs);
        as = warp_max(as);
        bs = warp_max(bs);
        if (lane == 0) {
          const double U1 = mul2(sh.U, emin);
          const int z1 = protect_update(U1, as, zs, omega);
          const double zs1 = mul2(zs, z1);
          const double U2 = mul2(U1, z1) + as * zs1;
          const int z2 = protect_update(U2, zs1, bs, omega);
          const int g = emin + z1 + z2;
          sh.U = mul2(U2, z2) + mul2(zs1, z2) * bs;
          sh.e_diag += g;
          sh.g = g;
          if (g != 0) ++local_scale_events;
        }
        __syncwarp();
        const int g = sh.g;
        for (int lb = lb_lo + lane; lb <= lb_hi; lb += 32) {
          const int sc = g - sh.pe[lb];
          if (sc != 0)
            for (int u = 0; u < 4; ++u) sh.zbuf[lb][u] = mul2(sh.zbuf[lb][u], sc);
        }
      }
      __syncthreads();
    }
    const int g = ROBUST ? sh.g : 0;
    // Phase C: every owned element takes its scale and this step's contributions.
    if (row_ok) {
      for (int c = my_c0; c < nt; c += CSTEP) {
        const int lbc = sh.colblk[c];
        const int dd = dr + lbc;
        T* yp = &Ys[my_r + c * LDY];
        if (dd == s) {
          const int cb0 = sh.bstart[lbc];
          *yp = static_cast<T>(sh.zbuf[lbc][(my_r - ra_r) + ma_r * (c - cb0)]);
          continue;
        }
        double y = static_cast<double>(*yp);
        if (ROBUST && g != 0) y = mul2(y, g);
        if (dd > s) {
          if (s >= lbc && s - lbc < dr) {  // block (kbs, lbc) below this row, solved now
            const int kbs = pb - 1 - (s - lbc);
            const int rs0 = sh.astart[kbs], mas = sh.astart[kbs + 1] - rs0;
            const int cb0 = sh.bstart[lbc];
            for (int ii = 0; ii < mas; ++ii)
              y = fma(-static_cast<double>(Ak[my_r + (rs0 + ii) * LDY]),
                      sh.zbuf[lbc][ii + mas * (c - cb0)], y);
          }
          if (s >= dr && s - dr < lbc) {  // block (kb_r, lbs) left of this column, solved now
            const int lbs = s - dr;
            const int cs0 = sh.bstart[lbs], nbs = sh.bstart[lbs + 1] - cs0;
            for (int jj = 0; jj < nbs; ++jj)
              y = fma(-sh.zbuf[lbs][(my_r - ra_r) + ma_r * jj],
                      static_cast<double>(Bk[(cs0 + jj) + c * LDY]), y);
          }
        }
        *yp = static_cast<T>(y);
      }
    }
    __syncthreads();
  }
  if (near) atomicOr(&sh.flags, kFlagNearSingular);
  if (local_scale_events) atomicAdd(&sh.nscale, local_scale_events);
}

// ----------------------------------------------------------------------------
// GEMM operand staging: L (rows x kdim) from column-major P (coalesced along rows),
// R (kdim x cols) from column-major P (coalesced along k); both stored k-major.
template <int TT, typename T, bool FROM_Y>
__device__ __forceinline__ void stage_left(T* L, const T* P, int64_t ld, int rows, int kdim) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
  for (int idx = threadIdx.x; idx < TT * TT; idx += kThreads) {
    const int r = idx % TT, kk = idx / TT;
    T v = T(0);
    if (r < rows && kk < kdim) {
      const T* src = P + r + kk * ld;
      v = FROM_Y ? __ldcg(src) : __ldg(src);
    }
    L[kk * LDG + r] = v;
  }
}
template <int TT, typename T, bool FROM_Y>
__device__ __forceinline__ void stage_right(T* R, const T* P, int64_t ld, int kdim, int cols) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
  for (int idx = threadIdx.x; idx < TT * TT; idx += kThreads) {
    const int kk = idx % TT, c = idx / TT;
    T v = T(0);
    if (kk < kdim && c < cols) {
      const T* src = P + kk + c * ld;
      v = FROM_Y ? __ldcg(src) : __ldg(src);
    }
    R[kk * LDG + c] = v;
  }
}

// acc -= L * R over kk < kdim; thread (tx, ty) owns rows tx*MR.., columns ty*NR..
template <int TT, typename T, int MR, int NR>
__device__ __forceinline__ void gemm_sub(T (&acc)[MR][NR], const T* L, const T* R, int kdim, int rbase,
                                         int cbase) {
  constexpr int LDG = DagSmem<TT, T>::LDG;
#pragma unroll 4
  for (int kk = 0; kk < kdim; ++kk) {
    T a[MR], b[NR];
#pragma unroll
    for (int i = 0; i < MR; ++i) a[i] = L[kk * LDG + rbase + i];
#pragma unroll
    for (int j = 0; j < NR; ++j) b[j] = R[kk * LDG + cbase + j];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
  }
}

template <int TT, typename T, bool ROBUST>
__global__ void __launch_bounds__(kThreads) dag_kernel(Work w) {
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

  for (;;) {
    if (tid == 0) {
      const int tk = atomicAdd(&ctrl->ticket, 1);
      sh.task = (tk < ctrl->ntasks && ld_volatile(&ctrl->err) == 0) ? tk : -1;
      sh.abort = 0;
      sh.flags = 0;
      sh.nscale = 0;
    }
    __syncthreads();
    if (sh.task < 0) break;
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
    int32_t* tflag = w.tflag + I.tile;
    double* tnorm = w.tnorm + I.tile;

    // ---- accumulator <- C_kl, exact infinity norm
    T acc[MR][NR];
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
      for (int r = tid; r < mt; r += kThreads) {
        double s = 0.0;
        for (int c = 0; c < nt; ++c) s += fabs(static_cast<double>(sh.Y[r + c * LDY]));
        atomic_max_nonneg(&sh.umax, s);
      }
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

    // ---- incoming updates, producers in anti-diagonal order
    const int d = (p - 1 - k) + l;
    const int s_lo = min(l, p - 1 - k);
    for (int s = s_lo; s < d && !sh.abort; ++s) {
      for (int side = 0; side < 2; ++side) {
        int prod;  // producer tile index
        int kdim;
        if (side == 0) {
          if (s < l) continue;
          const int i = p - 1 + l - s;  // A side: Y_kl -= A_ki Y_il
          prod = i * I.qmax + l;
          kdim = rb[i + 1] - rb[i];
        } else {
          if (s < p - 1 - k) continue;
          const int j = s - (p - 1 - k);  // B side: Y_kl -= Y_kj B_jl
          prod = k * I.qmax + j;
          kdim = cb[j + 1] - cb[j];
        }
        if (tid == 0) {
          if (!wait_flag(&tflag[prod], ctrl, w.timeout_ns)) sh.abort = 1;
        }
        __syncthreads();
        if (sh.abort) break;
        if (side == 0) {
          const int i = prod / I.qmax;
          stage_left<TT, T, false>(sh.L, A + r0 + (int64_t)rb[i] * I.lda, I.lda, mt, kdim);
          stage_right<TT, T, true>(sh.R, C + rb[i] + (int64_t)c0 * I.ldc, I.ldc, kdim, nt);
        } else {
          const int j = prod % I.qmax;
          stage_left<TT, T, true>(sh.L, C + r0 + (int64_t)cb[j] * I.ldc, I.ldc, mt, kdim);
          stage_right<TT, T, false>(sh.R, B + cb[j] + (int64_t)c0 * I.ldb, I.ldb, kdim, nt);
        }
        if (ROBUST && tid == 0) {
          const int ep = texp[prod];
          const double yp = tnorm[prod];
          const double on = (side == 0) ? an[(int64_t)k * I.pmax + prod / I.qmax]
                                        : bn[(int64_t)(prod % I.qmax) * I.qmax + l];
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
          if (sop != 0) {  // scale the Y operand (R on the A side, L on the B side)
            T* Yop = (side == 0) ? sh.R : sh.L;
            for (int idx = tid; idx < TT * DagSmem<TT, T>::LDG; idx += kThreads) Yop[idx] = mul2(Yop[idx], sop);
            __syncthreads();
          }
          if (sacc != 0) {
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
              for (int j = 0; j < NR; ++j) acc[i][j] = mul2(acc[i][j], sacc);
          }
        }
        gemm_sub<TT, T, MR, NR>(acc, sh.L, sh.R, kdim, rbase, cbase);
        __syncthreads();
      }
    }
    if (sh.abort) break;

    // ---- diagonal problem A_kk Z + Z B_ll = beta Y_kl
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < NR; ++j) sh.Y[(rbase + i) + (cbase + j) * LDY] = acc[i][j];
    for (int idx = tid; idx < TT * TT; idx += kThreads) {
      const int r = idx % TT, c = idx / TT;
      sh.L[r + c * LDY] = (r < mt && c < mt && r <= c + 1) ? __ldg(&A[(r0 + r) + (int64_t)(r0 + c) * I.lda]) : T(0);
      sh.R[r + c * LDY] = (r < nt && c < nt && r <= c + 1) ? __ldg(&B[(c0 + r) + (int64_t)(c0 + c) * I.ldb]) : T(0);
    }
    __syncthreads();
    diag_solve<TT, T, ROBUST>(sh, mt, nt, omega, st->smin);

    // ---- exact norm of the final tile, write back, publish
    if (tid == 0) sh.umax = 0ull;
    __syncthreads();
    for (int r = tid; r < mt; r += kThreads) {
      double s = 0.0;
      for (int c = 0; c < nt; ++c) s += fabs(static_cast<double>(sh.Y[r + c * LDY]));
      atomic_max_nonneg(&sh.umax, s);
    }
    for (int idx = tid; idx < mt * nt; idx += kThreads) {
      const int r = idx % mt, c = idx / mt;
      C[(r0 + r) + (int64_t)(c0 + c) * I.ldc] = sh.Y[r + c * LDY];
    }
    __syncthreads();
    if (tid == 0) {
      const double nrm = __longlong_as_double(static_cast<long long>(sh.umax));
      const int e = ROBUST ? sh.e_acc + sh.e_diag : 0;
      texp[task.tile] = e;
      tnorm[task.tile] = nrm;
      int fl = sh.flags;
      if (!(nrm <= 1.7976931348623157e308)) fl |= kFlagNonfiniteOut;
      if (fl) atomicOr(&st->flags, fl);
      if (ROBUST) {
        atomicMin(&st->minexp, e);
        if (sh.nscale) atomicAdd(&st->nscale, sh.nscale);
      }
      __threadfence();
      st_release(&tflag[task.tile], 1);
    }
    __syncthreads();
  }
}

}  // namespace sylv
