/*
 * sylv_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU oracle for the triangular Sylvester
 * equation  A*Y + Y*B = alpha*C  (Schwarz & Kjelgaard Mikkelsen, "Robust
 * Task-Parallel Solution of the Triangular Sylvester Equation", 2019).
 * A (m x m) and B (n x n) are upper quasi-triangular (real Schur form, Sec. 1,
 * eq. (4)): upper triangular except for 2x2 diagonal blocks marked by a nonzero
 * first subdiagonal entry.  All matrices are column-major.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this file's library.  The GPU library shares no code with it.
 *
 * What it computes:
 *   - oracle_protect_update / oracle_protect_division: power-of-two versions of
 *     the ProtectUpdate and ProtectDivision contracts of Sec. 2.1.
 *   - oracle_small_solve: the robust solve of a <=2x2 by <=2x2 Sylvester block
 *     through its <=4x4 Kronecker linear system by Gaussian elimination with
 *     complete pivoting (Sec. 2.1).
 *   - oracle_trsyl: Algorithm 2 (RobustSyl, global scale factor, robust != 0) or
 *     Algorithm 1 (no scaling, robust == 0), looping over the 1x1/2x2 diagonal
 *     blocks of A and B in the order the algorithms state (block column l
 *     ascending, block row k descending).
 *
 * Scale factors are carried as integer base-2 exponents: alpha = 2^log2scale,
 * so the scale never underflows even where a double alpha would.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS 0x1p-52        /* relative machine precision (spacing of doubles at 1) */
#define ORC_SMALLNUM 0x1p-1022 /* smallest normal double */

/* floor(log2(v)) for a positive finite double, via frexp: v = f*2^e, f in [0.5,1). */
static int floor_log2(double v) {
  int e;
  (void)frexp(v, &e);
  return e - 1;
}

/* ceil(log2(v)) for a positive finite double. */
static int ceil_log2(double v) {
  int e;
  double f = frexp(v, &e);
  return (f == 0.5) ? e - 1 : e;
}

/*
 * ProtectUpdate (Sec. 2.1): given upper bounds c = ||C||, t = ||A||, x = ||Y||, all
 * in [0, omega], return the base-2 exponent z <= 0 of a scale factor zeta = 2^z
 * with zeta*(c + t*x) <= omega exactly; no intermediate overflows.  zeta is the
 * largest power of two the contract allows, up to rounding: 2^-ceil(log2 u) with
 * u = (c + t*x)/omega, evaluated as c/omega + (t/omega)*x (omega is a power of two,
 * so both quotients are exact and nothing overflows) and enlarged by 2^-50 to
 * cover the two roundings.  The first test returns 1 when c + t*x <= omega holds
 * with a margin of four units of roundoff (a pass implies the exact inequality;
 * c == omega leaves no room for any nonzero t*x).
 */
int oracle_protect_update(double c, double t, double x, double omega) {
  const double shrink = 1.0 - 0x1p-51;
  if (t == 0.0 || x == 0.0) return 0; /* no update term: c <= omega already */
  if (x <= 1.0) {
    double lim = (omega - c) * shrink;
    if (lim > 0.0 && t * x <= lim) return 0;
  } else {
    if (t <= ((omega - c) / x) * shrink) return 0;
  }
  double u = c / omega + (t / omega) * x;
  int z = -ceil_log2(u * (1.0 + 0x1p-50));
  return z < 0 ? z : 0;
}

/*
 * ProtectDivision (Sec. 2.1): given |b| <= omega and a divisor magnitude d > 0,
 * return the exponent z <= 0 of zeta = 2^z such that zeta*|b|/d <= omega.
 * Only a divisor below one can enlarge |b|; then zeta is the largest power of
 * two not above d*omega/|b|.  d*omega and b*2^z are exact (omega is a power of
 * two), so the candidate from the rounded quotient is corrected by exact
 * comparisons.
 */
int oracle_protect_division(double b, double d, double omega) {
  b = fabs(b);
  d = fabs(d);
  if (d < 1.0 && b > d * omega) {
    double lim = d * omega;
    int z = floor_log2(lim / b);
    while (z < 0 && ldexp(b, z + 1) <= lim) ++z;
    while (ldexp(b, z) > lim) --z;
    return z;
  }
  return 0;
}

/*
 * Robust solve of the small Sylvester equation  A11*Z + Z*B11 = beta*R  with
 * A11 ma x ma, B11 nb x nb (ma, nb in {1,2}), Sec. 2.1.  The system is written
 * as (I_nb (x) A11 + B11^T (x) I_ma) vec(Z) = beta vec(R) and solved by Gaussian
 * elimination with complete pivoting.  Each update of the right-hand side is
 * guarded by ProtectUpdate and each division by ProtectDivision; beta = 2^log2beta
 * is the product of the guards.  A pivot of magnitude below smin is replaced by
 * smin (near-singular system) and the return value is then 1, else 0.
 *
 * A11 is given column-major with leading dimension lda11, B11 likewise; R is
 * ma x nb column-major with leading dimension ldr and is overwritten by Z.
 * robust == 0 skips every guard (beta = 1), as in Algorithm 1.
 */
int oracle_small_solve(int ma, int nb, const double* A11, int lda11, const double* B11,
                       int ldb11, double* R, int ldr, double smin, double omega, int robust,
                       int* log2beta) {
  int s = ma * nb;
  double M[4][4];
  double r[4];
  int colperm[4];
  int info = 0;
  int lb = 0;

  for (int u = 0; u < s; ++u) {
    int i = u % ma, j = u / ma;
    r[u] = R[i + (size_t)ldr * j];
    colperm[u] = u;
    for (int v = 0; v < s; ++v) {
      int i2 = v % ma, j2 = v / ma;
      double e = 0.0;
      if (j == j2) e += A11[i + (size_t)lda11 * i2];
      if (i == i2) e += B11[j2 + (size_t)ldb11 * j];
      M[u][v] = e;
    }
  }

  /* Forward elimination with complete pivoting. */
  for (int step = 0; step < s; ++step) {
    int pr = step, pc = step;
    double best = -1.0;
    for (int u = step; u < s; ++u)
      for (int v = step; v < s; ++v)
        if (fabs(M[u][v]) > best) {
          best = fabs(M[u][v]);
          pr = u;
          pc = v;
        }
    if (pr != step) {
      for (int v = 0; v < s; ++v) {
        double tmp = M[step][v];
        M[step][v] = M[pr][v];
        M[pr][v] = tmp;
      }
      double tmp = r[step];
      r[step] = r[pr];
      r[pr] = tmp;
    }
    if (pc != step) {
      for (int u = 0; u < s; ++u) {
        double tmp = M[u][step];
        M[u][step] = M[u][pc];
        M[u][pc] = tmp;
      }
      int t = colperm[step];
      colperm[step] = colperm[pc];
      colperm[pc] = t;
    }
    if (fabs(M[step][step]) < smin) {
      M[step][step] = smin;
      info = 1;
    }
    for (int u = step + 1; u < s; ++u) {
      double l = M[u][step] / M[step][step]; /* |l| <= 1 by complete pivoting */
      for (int v = step + 1; v < s; ++v) M[u][v] -= l * M[step][v];
      M[u][step] = 0.0;
      if (robust) {
        int z = oracle_protect_update(fabs(r[u]), fabs(l), fabs(r[step]), omega);
        if (z < 0) {
          for (int w = 0; w < s; ++w) r[w] = ldexp(r[w], z);
          lb += z;
        }
      }
      r[u] -= l * r[step];
    }
  }

  /* Back substitution; r holds the solved unknowns from position i+1 on. */
  for (int i = s - 1; i >= 0; --i) {
    for (int v = i + 1; v < s; ++v) {
      if (robust) {
        int z = oracle_protect_update(fabs(r[i]), fabs(M[i][v]), fabs(r[v]), omega);
        if (z < 0) {
          for (int w = 0; w < s; ++w) r[w] = ldexp(r[w], z);
          lb += z;
        }
      }
      r[i] -= M[i][v] * r[v];
    }
    if (robust) {
      int z = oracle_protect_division(r[i], M[i][i], omega);
      if (z < 0) {
        for (int w = 0; w < s; ++w) r[w] = ldexp(r[w], z);
        lb += z;
      }
    }
    r[i] = r[i] / M[i][i];
  }

  /* Undo the column permutation: unknown colperm[u] sits at position u. */
  double x[4];
  for (int u = 0; u < s; ++u) x[colperm[u]] = r[u];
  for (int u = 0; u < s; ++u) R[(u % ma) + (size_t)ldr * (u / ma)] = x[u];
  *log2beta = lb;
  return info;
}

/*
 * Partition an upper quasi-triangular matrix into its 1x1 and 2x2 diagonal
 * blocks (Sec. 1, eq. (4)): a nonzero T[i+1,i] starts a 2x2 block at i.
 * Writes the block start indices to starts[0..nblk-1] and starts[nblk] = n.
 * Returns nblk, or -1 if two consecutive subdiagonal entries are nonzero (not
 * quasi-triangular).
 */
int oracle_blocks(int64_t n, const double* T, int64_t ldt, int64_t* starts) {
  int64_t nb = 0, i = 0;
  while (i < n) {
    starts[nb++] = i;
    if (i + 1 < n && T[(i + 1) + ldt * i] != 0.0) {
      if (i + 2 < n && T[(i + 2) + ldt * (i + 1)] != 0.0) return -1;
      i += 2;
    } else {
      i += 1;
    }
  }
  starts[nb] = n;
  return (int)nb;
}

/* max over rows r0..r1-1 of sum over columns c0..c1-1 of |M[r,c]| (the infinity norm). */
static double inf_norm(const double* M, int64_t ld, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  double best = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    double s = 0.0;
    for (int64_t c = c0; c < c1; ++c) s += fabs(M[r + ld * c]);
    if (s > best) best = s;
  }
  return best;
}

/* Largest magnitude in a rectangle; NaN-propagating through *nan_seen. */
static double max_abs(const double* M, int64_t ld, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                      int* nan_seen) {
  double best = 0.0;
  for (int64_t c = c0; c < c1; ++c)
    for (int64_t r = r0; r < r1; ++r) {
      double v = fabs(M[r + ld * c]);
      if (v != v) *nan_seen = 1;
      if (v > best) best = v;
    }
  return best;
}

static void scale_all(double* Y, int64_t ldy, int64_t m, int64_t n, int z) {
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < m; ++r) Y[r + ldy * c] = ldexp(Y[r + ldy * c], z);
}

/*
 * Algorithm 2 (RobustSyl, robust != 0) or Algorithm 1 (robust == 0) on the whole
 * m x n problem, with the 1x1/2x2 diagonal blocks of A and B as the blocks.
 *
 *   Y <- C, alpha <- 1
 *   for l = 1..q (ascending), k = p..1 (descending):
 *     solve A_kk Z + Z B_ll = beta Y_kl robustly;        Y <- beta Y; Y_kl <- Z
 *     g1 = ProtectUpdate(||Y_{1:k-1,l}||, ||A_{1:k-1,k}||, ||Y_kl||);  Y <- g1 Y
 *     Y_{1:k-1,l} -= A_{1:k-1,k} Y_kl
 *     g2 = ProtectUpdate(max_{j>l} ||Y_kj||, ||Y_kl||, max_{j>l} ||B_lj||); Y <- g2 Y
 *     Y_{k,l+1:q} -= Y_kl B_{l,l+1:q}
 *     alpha <- alpha beta g1 g2
 *
 * The printed algorithm's last update reads B_{l,j+1:q}; the block row of B to
 * the right of the diagonal block, B_{l,l+1:q}, is the one the equation needs.
 *
 * C (ldc) is overwritten by Y; *log2scale receives log2(alpha) (an integer, since
 * every factor is a power of two).  smin is the pivot floor of the small solves.
 * *peak receives the largest magnitude any entry of Y held at any point (the
 * "Ensure" clause of Algorithm 2 is *peak <= omega); *nan_seen is set if an
 * entry became NaN.  Returns 0, 1 (a small solve was near singular and was
 * perturbed), or a negative value: -2 (A not quasi-triangular), -4 (B not
 * quasi-triangular), -99 (allocation failure).
 */
int oracle_trsyl(int64_t m, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double* C, int64_t ldc, double smin, double omega, int robust, int64_t* log2scale,
                 double* peak, int* nan_seen) {
  int64_t* as = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t* bs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int info = 0;
  int64_t e_alpha = 0;
  double pk = 0.0;
  int nan_flag = 0;
  if (!as || !bs) {
    free(as);
    free(bs);
    return -99;
  }
  int pb = oracle_blocks(m, A, lda, as);
  int qb = oracle_blocks(n, B, ldb, bs);
  if (pb < 0 || qb < 0) {
    free(as);
    free(bs);
    return pb < 0 ? -2 : -4;
  }
  double* Y = C;
  int64_t ldy = ldc;
  pk = max_abs(Y, ldy, 0, m, 0, n, &nan_flag);

  for (int l = 0; l < qb; ++l) {
    int64_t c0 = bs[l], c1 = bs[l + 1];
    for (int k = pb - 1; k >= 0; --k) {
      int64_t r0 = as[k], r1 = as[k + 1];
      int ma = (int)(r1 - r0), nbk = (int)(c1 - c0);

      /* Small solve of A_kk Z + Z B_ll = beta Y_kl; Z overwrites Y_kl. */
      int lbeta = 0;
      int sinfo = oracle_small_solve(ma, nbk, &A[r0 + lda * r0], (int)lda, &B[c0 + ldb * c0],
                                     (int)ldb, &Y[r0 + ldy * c0], (int)ldy, smin, omega, robust,
                                     &lbeta);
      if (sinfo) info = 1;
      if (lbeta < 0) {
        /* Y <- beta*Y everywhere except the block just solved, which already is beta-scaled. */
        double save[4];
        for (int u = 0; u < ma * nbk; ++u) save[u] = Y[r0 + (u % ma) + ldy * (c0 + u / ma)];
        scale_all(Y, ldy, m, n, lbeta);
        for (int u = 0; u < ma * nbk; ++u) Y[r0 + (u % ma) + ldy * (c0 + u / ma)] = save[u];
        e_alpha += lbeta;
      }
      {
        double v = max_abs(Y, ldy, r0, r1, c0, c1, &nan_flag);
        if (v > pk) pk = v;
      }

      /* Column update: Y_{1:k-1,l} -= A_{1:k-1,k} Y_kl. */
      if (r0 > 0) {
        if (robust) {
          double cn = inf_norm(Y, ldy, 0, r0, c0, c1);
          double an = inf_norm(A, lda, 0, r0, r0, r1);
          double yn = inf_norm(Y, ldy, r0, r1, c0, c1);
          int g1 = oracle_protect_update(cn, an, yn, omega);
          if (g1 < 0) {
            scale_all(Y, ldy, m, n, g1);
            e_alpha += g1;
          }
        }
        for (int64_t c = c0; c < c1; ++c)
          for (int64_t kk = r0; kk < r1; ++kk) {
            double z = Y[kk + ldy * c];
            const double* acol = &A[lda * kk];
            double* ycol = &Y[ldy * c];
            for (int64_t i = 0; i < r0; ++i) ycol[i] -= acol[i] * z;
          }
        double v = max_abs(Y, ldy, 0, r0, c0, c1, &nan_flag);
        if (v > pk) pk = v;
      }

      /* Row update: Y_{k,l+1:q} -= Y_kl B_{l,l+1:q}. */
      if (c1 < n) {
        if (robust) {
          double cn = 0.0, bn = 0.0;
          for (int j = l + 1; j < qb; ++j) {
            double a1 = inf_norm(Y, ldy, r0, r1, bs[j], bs[j + 1]);
            double b1 = inf_norm(B, ldb, c0, c1, bs[j], bs[j + 1]);
            if (a1 > cn) cn = a1;
            if (b1 > bn) bn = b1;
          }
          double yn = inf_norm(Y, ldy, r0, r1, c0, c1);
          int g2 = oracle_protect_update(cn, yn, bn, omega);
          if (g2 < 0) {
            scale_all(Y, ldy, m, n, g2);
            e_alpha += g2;
          }
        }
        for (int64_t j = c1; j < n; ++j)
          for (int64_t kk = c0; kk < c1; ++kk) {
            double b = B[kk + ldb * j];
            for (int64_t r = r0; r < r1; ++r) Y[r + ldy * j] -= Y[r + ldy * kk] * b;
          }
        double v = max_abs(Y, ldy, r0, r1, c1, n, &nan_flag);
        if (v > pk) pk = v;
      }
    }
  }
  free(as);
  free(bs);
  *log2scale = e_alpha;
  *peak = pk;
  *nan_seen = nan_flag;
  return info;
}
