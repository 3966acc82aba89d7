/*
 * Plain FP64 CPU oracle for ILU0-preconditioned BiCGStab on 3x3 block-CSR
 * matrices.  TEST INFRASTRUCTURE ONLY: the GPU library never links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: single-threaded loops, no blocking, no fusion, no reordering beyond what
 * each definition states.  Compiled with -O2 -ffp-contract=off so that no
 * multiply-add is fused.
 *
 * Storage convention (Section 4.1 on contiguous blocks; Section 4.7, figure
 * "Memory layout of blocks in OPM (left) and amgcl (right)", left panel):
 * block-CSR with nb block rows, rowptr[nb+1], colidx[nnzb]
 * sorted and unique inside every row, and each 3x3 block stored contiguously
 * and row-major: entry (r, c) of block m is vals[9*m + 3*r + c].  Vectors are
 * nb*3 doubles, the 3 unknowns of one cell contiguous (Section 4.1).
 *
 * Pins: every function below is checked by the CPU test suite against
 * something other than itself (dense brute force, exact LU on no-fill
 * patterns, the ILU0 defining identity, closed forms of grid schedules).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BS 3
#define BS2 9

/* ------------------------------------------------------------------------ */
/* small dense helpers on 3x3 row-major blocks                              */
/* ------------------------------------------------------------------------ */

/* c = a * b */
static void blk_mul(const double *a, const double *b, double *c) {
  for (int r = 0; r < BS; ++r)
    for (int s = 0; s < BS; ++s) {
      double acc = 0.0;
      for (int t = 0; t < BS; ++t) acc += a[r * BS + t] * b[t * BS + s];
      c[r * BS + s] = acc;
    }
}

/* c -= a * b */
static void blk_mul_sub(const double *a, const double *b, double *c) {
  double p[BS2];
  blk_mul(a, b, p);
  for (int e = 0; e < BS2; ++e) c[e] -= p[e];
}

/* y += a * x (3-vector) */
static void blk_matvec_add(const double *a, const double *x, double *y) {
  for (int r = 0; r < BS; ++r) {
    double acc = 0.0;
    for (int c = 0; c < BS; ++c) acc += a[r * BS + c] * x[c];
    y[r] += acc;
  }
}

/*
 * Inverse of a 3x3 block by Gauss-Jordan elimination with partial pivoting
 * (textbook method; deliberately not the adjugate formula the GPU uses).
 * Returns 0, or -1 when a pivot is exactly zero or the result is not finite.
 */
int orc_inv3(const double *a_in, double *ainv) {
  double a[BS][2 * BS];
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      a[r][c] = a_in[r * BS + c];
      a[r][BS + c] = (r == c) ? 1.0 : 0.0;
    }
  for (int col = 0; col < BS; ++col) {
    int piv = col;
    for (int r = col + 1; r < BS; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return -1;
    if (piv != col)
      for (int c = 0; c < 2 * BS; ++c) {
        double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    double d = a[col][col];
    for (int c = 0; c < 2 * BS; ++c) a[col][c] /= d;
    for (int r = 0; r < BS; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      if (f != 0.0)
        for (int c = 0; c < 2 * BS; ++c) a[r][c] -= f * a[col][c];
    }
  }
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      ainv[r * BS + c] = a[r][BS + c];
      if (!isfinite(ainv[r * BS + c])) return -1;
    }
  return 0;
}

/* position of column j in row i, or -1 (linear scan: rows are short) */
static int64_t find_block(const int32_t *rowptr, const int32_t *colidx, int32_t i, int32_t j) {
  for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m)
    if (colidx[m] == j) return m;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Blocked SpMV, y = A x (Section 4.3): y_i = sum over the blocks A_ij of    */
/* row i, in colidx order, of the dense product A_ij x_j.                   */
/* ------------------------------------------------------------------------ */
void orc_spmv(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
              const double *x, double *y) {
  for (int32_t i = 0; i < nb; ++i) {
    double yi[BS] = {0.0, 0.0, 0.0};
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m)
      blk_matvec_add(vals + BS2 * m, x + (int64_t)BS * colidx[m], yi);
    for (int r = 0; r < BS; ++r) y[(int64_t)BS * i + r] = yi[r];
  }
}

/*
 * Standard-well contributions kept separate (Section 4.6, the algorithm
 * "adding the wellcontributions separately"): for every well, t1 = B x
 * (B: one row of 4x3 blocks, one per perforated cell), t2 = inv(D) t1 (D a
 * single 4x4 block, given inverted), y -= C^T t2.  Blocks row-major.
 */
void orc_apply_wells(int32_t nwells, const int32_t *wptr, const int32_t *wcells, const double *B,
                     const double *C, const double *Dinv, const double *x, double *y) {
  for (int32_t w = 0; w < nwells; ++w) {
    double t1[4] = {0.0, 0.0, 0.0, 0.0}, t2[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t p = wptr[w]; p < wptr[w + 1]; ++p)
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < BS; ++c) t1[r] += B[12 * (int64_t)p + 3 * r + c] * x[(int64_t)BS * wcells[p] + c];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) t2[r] += Dinv[16 * (int64_t)w + 4 * r + c] * t1[c];
    for (int32_t p = wptr[w]; p < wptr[w + 1]; ++p)
      for (int c = 0; c < BS; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 4; ++r) acc += C[12 * (int64_t)p + 3 * r + c] * t2[r];
        y[(int64_t)BS * wcells[p] + c] -= acc;
      }
  }
}

/* y = A x - sum over wells of C^T inv(D) B x */
void orc_spmv_wells(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                    int32_t nwells, const int32_t *wptr, const int32_t *wcells, const double *B,
                    const double *C, const double *Dinv, const double *x, double *y) {
  orc_spmv(nb, rowptr, colidx, vals, x, y);
  orc_apply_wells(nwells, wptr, wcells, B, C, Dinv, x, y);
}

/* ------------------------------------------------------------------------ */
/* ILU0 decomposition (Section 2.2, Algorithm 2), block version.            */
/*                                                                          */
/* Algorithm 2 eliminates pivot r = 0..nb-1 in turn: every row i > r that   */
/* has a block (i, r) in the pattern S gets a_ir <- a_ir * inv(a_rr), and   */
/* then a_ij <- a_ij - a_ir * a_rj for each j > r with (i,j) and (r,j) in S. */
/* For blocks the multiplier is a right product with the inverse pivot      */
/* block.  Here the same updates are applied row by row: for row i, its     */
/* pivots k < i are taken in ascending order, which gives every entry the    */
/* same updates in the same order as the pivot-by-pivot loop.               */
/*                                                                          */
/* Output: lu holds L (unit lower, strictly-lower blocks stored) and U      */
/* (diagonal and strictly-upper blocks) in the pattern of A; dinv[9*i] is   */
/* the inverse of U's diagonal block of row i.                              */
/* Returns 0, or -(1 + i) when the pivot block of row i is singular, or     */
/* -(1 + nb + i) when row i has no diagonal block.                          */
/* ------------------------------------------------------------------------ */
int orc_ilu0(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
             double *lu, double *dinv) {
  memcpy(lu, vals, sizeof(double) * BS2 * (size_t)rowptr[nb]);
  for (int32_t i = 0; i < nb; ++i) {
    for (int64_t mk = rowptr[i]; mk < rowptr[i + 1]; ++mk) {
      int32_t k = colidx[mk];
      if (k >= i) break; /* colidx is sorted: the rest is diagonal / upper */
      /* L_ik = A_ik * inv(U_kk) */
      double lik[BS2];
      blk_mul(lu + BS2 * mk, dinv + BS2 * (int64_t)k, lik);
      memcpy(lu + BS2 * mk, lik, sizeof lik);
      /* A_ij -= L_ik * U_kj for every j > k present in both row i and row k */
      for (int64_t mj = mk + 1; mj < rowptr[i + 1]; ++mj) {
        int32_t j = colidx[mj];
        int64_t mkj = find_block(rowptr, colidx, k, j);
        if (mkj >= 0) blk_mul_sub(lik, lu + BS2 * mkj, lu + BS2 * mj);
      }
    }
    int64_t md = find_block(rowptr, colidx, i, i);
    if (md < 0) return -(1 + nb + i);
    if (orc_inv3(lu + BS2 * md, dinv + BS2 * (int64_t)i) != 0) return -(1 + i);
  }
  return 0;
}

/*
 * Fine-grained iterative ILU0 of Chow & Patel (2015), the "Chow Patel ILU0"
 * of the paper's library table (Section 3): the factors are the fixed point
 * of, for every block (i,j) of the pattern at once (synchronous sweeps, all
 * right-hand sides from the previous sweep),
 *   s = A_ij - sum_{k < min(i,j)} L_ik U_kj      (k ascending),
 *   L_ij = s inv(U_jj) (i > j),  U_ii = s (its inverse kept),  U_ij = s (i < j).
 * Initial guess L_ij = A_ij inv(A_jj), U_ij = A_ij.  After enough sweeps it
 * reaches the ILU0 factors of orc_ilu0 with the same operations.  Output
 * and returns as orc_ilu0 (a singular pivot during any sweep fails).
 */
int orc_ilu0_cp(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals, int32_t sweeps,
                double *lu, double *dinv) {
  const size_t nnzb = (size_t)rowptr[nb];
  for (int32_t i = 0; i < nb; ++i) {
    int64_t md = find_block(rowptr, colidx, i, i);
    if (md < 0) return -(1 + nb + i);
    if (orc_inv3(vals + BS2 * md, dinv + BS2 * (int64_t)i) != 0) return -(1 + i);
  }
  for (int32_t i = 0; i < nb; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      if (colidx[m] < i) blk_mul(vals + BS2 * m, dinv + BS2 * (int64_t)colidx[m], lu + BS2 * m);
      else memcpy(lu + BS2 * m, vals + BS2 * m, sizeof(double) * BS2);
    }
  double *lu2 = malloc(sizeof(double) * BS2 * (nnzb ? nnzb : 1));
  double *d2 = malloc(sizeof(double) * BS2 * (size_t)(nb ? nb : 1));
  int status = 0;
  for (int32_t t = 0; t < sweeps && status == 0; ++t) {
    for (int32_t i = 0; i < nb && status == 0; ++i)
      for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
        const int32_t j = colidx[m];
        const int32_t lim = j < i ? j : i;
        double sum[BS2];
        memcpy(sum, vals + BS2 * m, sizeof sum);
        for (int64_t mk = rowptr[i]; mk < rowptr[i + 1] && colidx[mk] < lim; ++mk) {
          int64_t mkj = find_block(rowptr, colidx, colidx[mk], j);
          if (mkj >= 0) blk_mul_sub(lu + BS2 * mk, lu + BS2 * mkj, sum);
        }
        if (j < i) {
          blk_mul(sum, dinv + BS2 * (int64_t)j, lu2 + BS2 * m);
        } else {
          memcpy(lu2 + BS2 * m, sum, sizeof sum);
          if (j == i && orc_inv3(sum, d2 + BS2 * (int64_t)i) != 0) {
            status = -(1 + i);
            break;
          }
        }
      }
    if (status == 0) {
      memcpy(lu, lu2, sizeof(double) * BS2 * nnzb);
      memcpy(dinv, d2, sizeof(double) * BS2 * (size_t)nb);
    }
  }
  free(lu2);
  free(d2);
  return status;
}

/*
 * The triangular solves by Jacobi iteration (Anzt, Chow & Dongarra 2015):
 * `sweeps` synchronous sweeps for L y = r from y = r,
 *   y_i <- r_i - sum_{j<i} L_ij y_j,
 * then `sweeps` for U z = y from z_i = inv(U_ii) y_i,
 *   z_i <- inv(U_ii) (y_i - sum_{j>i} U_ij z_j),
 * every sweep reading the previous iterate.  Exact after as many sweeps as
 * the longest dependency chain of the factor.
 */
void orc_ilu_apply_jacobi(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *lu,
                          const double *dinv, const double *r, double *z, int32_t sweeps) {
  const size_t n = (size_t)BS * nb;
  double *y = malloc(sizeof(double) * (n ? n : 1)), *y2 = malloc(sizeof(double) * (n ? n : 1));
  double *z2 = malloc(sizeof(double) * (n ? n : 1));
  memcpy(y, r, sizeof(double) * n);
  for (int32_t t = 0; t < sweeps; ++t) {
    for (int32_t i = 0; i < nb; ++i) {
      double acc[BS];
      for (int c = 0; c < BS; ++c) acc[c] = r[(int64_t)BS * i + c];
      for (int64_t m = rowptr[i]; m < rowptr[i + 1] && colidx[m] < i; ++m) {
        double tv[BS] = {0.0, 0.0, 0.0};
        blk_matvec_add(lu + BS2 * m, y + (int64_t)BS * colidx[m], tv);
        for (int c = 0; c < BS; ++c) acc[c] -= tv[c];
      }
      memcpy(y2 + (int64_t)BS * i, acc, sizeof acc);
    }
    memcpy(y, y2, sizeof(double) * n);
  }
  for (int32_t i = 0; i < nb; ++i) {
    double zi[BS] = {0.0, 0.0, 0.0};
    blk_matvec_add(dinv + BS2 * (int64_t)i, y + (int64_t)BS * i, zi);
    memcpy(z + (int64_t)BS * i, zi, sizeof zi);
  }
  for (int32_t t = 0; t < sweeps; ++t) {
    for (int32_t i = 0; i < nb; ++i) {
      double acc[BS];
      for (int c = 0; c < BS; ++c) acc[c] = y[(int64_t)BS * i + c];
      for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
        if (colidx[m] <= i) continue;
        double tv[BS] = {0.0, 0.0, 0.0};
        blk_matvec_add(lu + BS2 * m, z + (int64_t)BS * colidx[m], tv);
        for (int c = 0; c < BS; ++c) acc[c] -= tv[c];
      }
      double zi[BS] = {0.0, 0.0, 0.0};
      blk_matvec_add(dinv + BS2 * (int64_t)i, acc, zi);
      memcpy(z2 + (int64_t)BS * i, zi, sizeof zi);
    }
    memcpy(z, z2, sizeof(double) * n);
  }
  free(y);
  free(y2);
  free(z2);
}

/* ------------------------------------------------------------------------ */
/* ILU0 application (Section 2.2, Algorithm 1, equations 3 and 4):          */
/* solve L y = r by forward substitution with the unit lower factor, then   */
/* U z = y by backward substitution.                                        */
/*   forward:  y_i = r_i - sum_{j<i} L_ij y_j,             i ascending      */
/*   backward: z_i = inv(U_ii) (y_i - sum_{j>i} U_ij z_j),  i descending     */
/* ------------------------------------------------------------------------ */
void orc_ilu_apply(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *lu,
                   const double *dinv, const double *r, double *z) {
  double *y = (double *)malloc(sizeof(double) * BS * (size_t)nb);
  for (int32_t i = 0; i < nb; ++i) {
    double acc[BS];
    for (int c = 0; c < BS; ++c) acc[c] = r[(int64_t)BS * i + c];
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j >= i) break;
      double t[BS] = {0.0, 0.0, 0.0};
      blk_matvec_add(lu + BS2 * m, y + (int64_t)BS * j, t);
      for (int c = 0; c < BS; ++c) acc[c] -= t[c];
    }
    for (int c = 0; c < BS; ++c) y[(int64_t)BS * i + c] = acc[c];
  }
  for (int32_t i = nb - 1; i >= 0; --i) {
    double acc[BS];
    for (int c = 0; c < BS; ++c) acc[c] = y[(int64_t)BS * i + c];
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j <= i) continue;
      double t[BS] = {0.0, 0.0, 0.0};
      blk_matvec_add(lu + BS2 * m, z + (int64_t)BS * j, t);
      for (int c = 0; c < BS; ++c) acc[c] -= t[c];
    }
    double zi[BS] = {0.0, 0.0, 0.0};
    blk_matvec_add(dinv + BS2 * (int64_t)i, acc, zi);
    for (int c = 0; c < BS; ++c) z[(int64_t)BS * i + c] = zi[c];
  }
  free(y);
}

/* ------------------------------------------------------------------------ */
/* Single-precision variant of the two functions above: the same steps in   */
/* float arithmetic, on values rounded to float.  Used as the reference for  */
/* the form that stores and runs the ILU0 factors in FP32.                   */
/* ------------------------------------------------------------------------ */
static int inv3_f(const float *a_in, float *ainv) {
  double a[BS2], o[BS2];
  for (int e = 0; e < BS2; ++e) a[e] = a_in[e];
  if (orc_inv3(a, o) != 0) return -1;
  for (int e = 0; e < BS2; ++e) ainv[e] = (float)o[e];
  return 0;
}

static void blk_mul_f(const float *a, const float *b, float *c) {
  for (int r = 0; r < BS; ++r)
    for (int s = 0; s < BS; ++s) {
      float acc = 0.0f;
      for (int t = 0; t < BS; ++t) acc += a[r * BS + t] * b[t * BS + s];
      c[r * BS + s] = acc;
    }
}

int orc_ilu0_f32(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                 float *lu, float *dinv) {
  size_t nnz = (size_t)rowptr[nb];
  for (size_t e = 0; e < BS2 * nnz; ++e) lu[e] = (float)vals[e];
  for (int32_t i = 0; i < nb; ++i) {
    for (int64_t mk = rowptr[i]; mk < rowptr[i + 1]; ++mk) {
      int32_t k = colidx[mk];
      if (k >= i) break;
      float lik[BS2];
      blk_mul_f(lu + BS2 * mk, dinv + BS2 * (int64_t)k, lik);
      memcpy(lu + BS2 * mk, lik, sizeof lik);
      for (int64_t mj = mk + 1; mj < rowptr[i + 1]; ++mj) {
        int64_t mkj = find_block(rowptr, colidx, k, colidx[mj]);
        if (mkj >= 0) {
          float p[BS2];
          blk_mul_f(lik, lu + BS2 * mkj, p);
          for (int e = 0; e < BS2; ++e) lu[BS2 * mj + e] -= p[e];
        }
      }
    }
    int64_t md = find_block(rowptr, colidx, i, i);
    if (md < 0) return -(1 + nb + i);
    if (inv3_f(lu + BS2 * md, dinv + BS2 * (int64_t)i) != 0) return -(1 + i);
  }
  return 0;
}

void orc_ilu_apply_f32(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const float *lu,
                       const float *dinv, const double *r, double *z) {
  float *y = (float *)malloc(sizeof(float) * BS * (size_t)nb);
  float *zf = (float *)malloc(sizeof(float) * BS * (size_t)nb);
  for (int32_t i = 0; i < nb; ++i) {
    float acc[BS];
    for (int c = 0; c < BS; ++c) acc[c] = (float)r[(int64_t)BS * i + c];
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j >= i) break;
      for (int a = 0; a < BS; ++a) {
        float t = 0.0f;
        for (int c = 0; c < BS; ++c) t += lu[BS2 * m + a * BS + c] * y[(int64_t)BS * j + c];
        acc[a] -= t;
      }
    }
    for (int c = 0; c < BS; ++c) y[(int64_t)BS * i + c] = acc[c];
  }
  for (int32_t i = nb - 1; i >= 0; --i) {
    float acc[BS];
    for (int c = 0; c < BS; ++c) acc[c] = y[(int64_t)BS * i + c];
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j <= i) continue;
      for (int a = 0; a < BS; ++a) {
        float t = 0.0f;
        for (int c = 0; c < BS; ++c) t += lu[BS2 * m + a * BS + c] * zf[(int64_t)BS * j + c];
        acc[a] -= t;
      }
    }
    for (int a = 0; a < BS; ++a) {
      float t = 0.0f;
      for (int c = 0; c < BS; ++c) t += dinv[BS2 * (int64_t)i + a * BS + c] * acc[c];
      zf[(int64_t)BS * i + a] = t;
    }
  }
  for (size_t e = 0; e < BS * (size_t)nb; ++e) z[e] = zf[e];
  free(y);
  free(zf);
}

/* ------------------------------------------------------------------------ */
/* BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput. 13(2), 1992), right  */
/* preconditioned by the ILU0 factors, x0 = 0, shadow residual r^ = r0.     */
/* Stopping rule (Section 4.2): relative reduction of the residual 2-norm   */
/* by rtol, at most maxit iterations; it is tested after each half step.    */
/* The preconditioner is either the FP64 factors (lu, dinv) or, when lu32   */
/* is not NULL, the FP32 ones (lu32, dinv32).                               */
/*                                                                          */
/* Returns 0 converged, 1 not converged after maxit, -5 breakdown           */
/* (rho, (r^,v), (t,t) or omega exactly zero), -6 non-finite rhs.           */
/* *iters = iterations begun (a half-step exit counts as its iteration);    */
/* *relres = true ||b - A x|| / ||b|| after the solve; res_hist (optional,  */
/* length 2*maxit+1) receives ||r0||, then ||s|| and ||r|| of each step.     */
/* ------------------------------------------------------------------------ */
static double dot(size_t n, const double *a, const double *b) {
  double s = 0.0;
  for (size_t e = 0; e < n; ++e) s += a[e] * b[e];
  return s;
}

/*
 * The same iteration with a preconditioner on its own pattern (mrowptr,
 * mcolidx): the block-Jacobi ILU0 of Section 4.5 factorises only the blocks
 * inside a partition while the SpMV keeps the whole matrix.
 */
int orc_bicgstab_x(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                   const int32_t *mrowptr, const int32_t *mcolidx, const double *lu, const double *dinv,
                   const float *lu32, const float *dinv32, int32_t nwells, const int32_t *wptr,
                   const int32_t *wcells, const double *B, const double *C, const double *Dinv, int32_t tri_sweeps,
                   const double *b, double *x, double rtol, int32_t maxit, int32_t *iters, double *relres,
                   double *res_hist);

int orc_bicgstab_w(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                   const int32_t *mrowptr, const int32_t *mcolidx, const double *lu, const double *dinv,
                   const float *lu32, const float *dinv32, int32_t nwells, const int32_t *wptr,
                   const int32_t *wcells, const double *B, const double *C, const double *Dinv, const double *b,
                   double *x, double rtol, int32_t maxit, int32_t *iters, double *relres, double *res_hist) {
  return orc_bicgstab_x(nb, rowptr, colidx, vals, mrowptr, mcolidx, lu, dinv, lu32, dinv32, nwells, wptr, wcells,
                        B, C, Dinv, 0, b, x, rtol, maxit, iters, relres, res_hist);
}

int orc_bicgstab_pc(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                    const int32_t *mrowptr, const int32_t *mcolidx, const double *lu, const double *dinv,
                    const float *lu32, const float *dinv32, const double *b, double *x, double rtol,
                    int32_t maxit, int32_t *iters, double *relres, double *res_hist) {
  return orc_bicgstab_w(nb, rowptr, colidx, vals, mrowptr, mcolidx, lu, dinv, lu32, dinv32, 0, NULL, NULL, NULL,
                        NULL, NULL, b, x, rtol, maxit, iters, relres, res_hist);
}

int orc_bicgstab(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                 const double *lu, const double *dinv, const float *lu32, const float *dinv32,
                 const double *b, double *x, double rtol, int32_t maxit, int32_t *iters,
                 double *relres, double *res_hist) {
  return orc_bicgstab_pc(nb, rowptr, colidx, vals, rowptr, colidx, lu, dinv, lu32, dinv32, b, x, rtol, maxit,
                         iters, relres, res_hist);
}

/*
 * The general form: preconditioner on its own pattern (block-Jacobi,
 * Section 4.5), standard wells applied separately in every product with
 * the system operator (Section 4.6; nwells = 0: none), and the triangular
 * solves by tri_sweeps Jacobi sweeps (0: exact substitution).  The
 * preconditioner is the ILU0 of the cell matrix only.
 */
int orc_bicgstab_x(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                   const int32_t *mrowptr, const int32_t *mcolidx, const double *lu, const double *dinv,
                   const float *lu32, const float *dinv32, int32_t nwells, const int32_t *wptr,
                   const int32_t *wcells, const double *B, const double *C, const double *Dinv, int32_t tri_sweeps,
                   const double *b, double *x, double rtol, int32_t maxit, int32_t *iters, double *relres,
                   double *res_hist) {
  size_t n = (size_t)BS * nb;
  double *r = calloc(n, sizeof(double)), *rh = calloc(n, sizeof(double));
  double *p = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
  double *ph = calloc(n, sizeof(double)), *s = calloc(n, sizeof(double));
  double *sh = calloc(n, sizeof(double)), *t = calloc(n, sizeof(double));
  int status = 1;
  *iters = 0;
  for (size_t e = 0; e < n; ++e) {
    x[e] = 0.0;
    r[e] = b[e];
    rh[e] = b[e];
  }
  double n0 = sqrt(dot(n, r, r));
  if (res_hist) res_hist[0] = n0;
  if (!isfinite(n0)) {
    status = -6;
    goto done;
  }
  if (n0 == 0.0) {
    status = 0;
    goto done;
  }
  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  double tol = rtol * n0;
  for (int32_t k = 1; k <= maxit; ++k) {
    *iters = k;
    double rho = dot(n, rh, r);
    if (rho == 0.0) {
      status = -5;
      break;
    }
    double beta = (rho / rho_prev) * (alpha / omega);
    for (size_t e = 0; e < n; ++e) p[e] = r[e] + beta * (p[e] - omega * v[e]);
    if (lu32) orc_ilu_apply_f32(nb, mrowptr, mcolidx, lu32, dinv32, p, ph);
    else if (tri_sweeps > 0) orc_ilu_apply_jacobi(nb, mrowptr, mcolidx, lu, dinv, p, ph, tri_sweeps);
    else orc_ilu_apply(nb, mrowptr, mcolidx, lu, dinv, p, ph);
    orc_spmv_wells(nb, rowptr, colidx, vals, nwells, wptr, wcells, B, C, Dinv, ph, v);
    double rhv = dot(n, rh, v);
    if (rhv == 0.0) {
      status = -5;
      break;
    }
    alpha = rho / rhv;
    for (size_t e = 0; e < n; ++e) s[e] = r[e] - alpha * v[e];
    double ns = sqrt(dot(n, s, s));
    if (res_hist) res_hist[2 * k - 1] = ns;
    if (ns <= tol) { /* half-step exit */
      for (size_t e = 0; e < n; ++e) x[e] += alpha * ph[e];
      status = 0;
      break;
    }
    if (lu32) orc_ilu_apply_f32(nb, mrowptr, mcolidx, lu32, dinv32, s, sh);
    else if (tri_sweeps > 0) orc_ilu_apply_jacobi(nb, mrowptr, mcolidx, lu, dinv, s, sh, tri_sweeps);
    else orc_ilu_apply(nb, mrowptr, mcolidx, lu, dinv, s, sh);
    orc_spmv_wells(nb, rowptr, colidx, vals, nwells, wptr, wcells, B, C, Dinv, sh, t);
    double tt = dot(n, t, t);
    if (tt == 0.0) {
      status = -5;
      break;
    }
    omega = dot(n, t, s) / tt;
    if (omega == 0.0) {
      status = -5;
      break;
    }
    for (size_t e = 0; e < n; ++e) {
      x[e] += alpha * ph[e] + omega * sh[e];
      r[e] = s[e] - omega * t[e];
    }
    rho_prev = rho;
    double nr = sqrt(dot(n, r, r));
    if (res_hist) res_hist[2 * k] = nr;
    if (nr <= tol) {
      status = 0;
      break;
    }
  }
done:
  if (status == -6) {
    *relres = NAN;
  } else if (n0 == 0.0) {
    *relres = 0.0;
  } else {
    orc_spmv_wells(nb, rowptr, colidx, vals, nwells, wptr, wcells, B, C, Dinv, x, t);
    double nres = 0.0;
    for (size_t e = 0; e < n; ++e) nres += (b[e] - t[e]) * (b[e] - t[e]);
    *relres = sqrt(nres) / n0;
  }
  free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  return status;
}

/*
 * Restarted GMRES(m) (Saad & Schultz 1986), OPM's other Krylov solver
 * (Section 2), right-preconditioned by the ILU0 factors, x0 = 0.  Arnoldi
 * with classical Gram-Schmidt applied twice (each pass: all projections
 * h = V^T w first, then w -= V h); Givens rotations keep the least-squares
 * problem triangular; the estimate |g_{j+1}| of ||r|| is tested after every
 * step against rtol ||r_0|| (the rule of Section 4.2).  At the end of a
 * cycle (m steps, convergence, maxit or an exact breakdown) x += inv(M) V y
 * with H y = g; a new cycle starts from the true residual b - A x.  iters
 * counts Arnoldi steps over all cycles.  Returns 0 (converged),
 * 1 (maxit reached), -5 (breakdown: a zero rotation denominator), -6
 * (non-finite b or residual estimate; x then holds the last cycle's start).  res_hist (optional, maxit + 1
 * entries): ||r_0||, then the estimate after each step.
 */
int orc_gmres(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals, const double *lu,
              const double *dinv, const double *b, double *x, double rtol, int32_t maxit, int32_t restart,
              int32_t *iters, double *relres, double *res_hist) {
  const size_t n = (size_t)BS * nb;
  const int m = restart > 0 ? restart : 30;
  double *V = calloc((size_t)(m + 1) * n, sizeof(double));
  double *w = calloc(n, sizeof(double)), *z = calloc(n, sizeof(double)), *r = calloc(n, sizeof(double));
  double *H = calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i * m + j] */
  double *cs = calloc((size_t)m, sizeof(double)), *sn = calloc((size_t)m, sizeof(double));
  double *g = calloc((size_t)m + 1, sizeof(double)), *y = calloc((size_t)m, sizeof(double));
  double *h1 = calloc((size_t)m + 1, sizeof(double)), *h2 = calloc((size_t)m + 1, sizeof(double));
  int status = 1;
  *iters = 0;
  for (size_t e = 0; e < n; ++e) {
    x[e] = 0.0;
    r[e] = b[e];
  }
  const double n0 = sqrt(dot(n, r, r));
  double beta = n0;
  if (res_hist) res_hist[0] = n0;
  if (!isfinite(n0)) {
    status = -6;
    goto done;
  }
  if (n0 == 0.0) {
    status = 0;
    goto done;
  }
  const double tol = rtol * n0;
  int32_t k = 0;
  for (;;) {
    for (size_t e = 0; e < n; ++e) V[e] = r[e] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int j = 0, conv = 0;
    for (; j < m && k < maxit; ++j) {
      ++k;
      orc_ilu_apply(nb, rowptr, colidx, lu, dinv, V + (size_t)j * n, z);
      orc_spmv(nb, rowptr, colidx, vals, z, w);
      for (int i = 0; i <= j; ++i) h1[i] = dot(n, V + (size_t)i * n, w);
      for (size_t e = 0; e < n; ++e) {
        double acc = 0.0;
        for (int i = 0; i <= j; ++i) acc += h1[i] * V[(size_t)i * n + e];
        w[e] -= acc;
      }
      for (int i = 0; i <= j; ++i) h2[i] = dot(n, V + (size_t)i * n, w);
      for (size_t e = 0; e < n; ++e) {
        double acc = 0.0;
        for (int i = 0; i <= j; ++i) acc += h2[i] * V[(size_t)i * n + e];
        w[e] -= acc;
      }
      for (int i = 0; i <= j; ++i) H[i * m + j] = h1[i] + h2[i];
      const double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (size_t e = 0; e < n; ++e) V[(size_t)(j + 1) * n + e] = w[e] / hn;
      for (int i = 0; i < j; ++i) { /* earlier rotations on column j */
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[j * m + j], c = H[(j + 1) * m + j];
      const double den = sqrt(a * a + c * c);
      if (den == 0.0) { /* w = 0 with H_jj = 0: no progress possible */
        status = -5;
        goto stop;
      }
      cs[j] = a / den;
      sn[j] = c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (res_hist) res_hist[k] = fabs(g[j + 1]);
      if (!isfinite(g[j + 1])) {
        status = -6;
        goto stop;
      }
      if (fabs(g[j + 1]) <= tol || hn == 0.0) {
        conv = 1;
        ++j;
        break;
      }
    }
    /* x += inv(M) V y, H y = g (back substitution over the j steps done) */
    for (int i = j - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < j; ++l) acc -= H[i * m + l] * y[l];
      y[i] = acc / H[i * m + i];
    }
    for (size_t e = 0; e < n; ++e) {
      double acc = 0.0;
      for (int i = 0; i < j; ++i) acc += y[i] * V[(size_t)i * n + e];
      w[e] = acc;
    }
    orc_ilu_apply(nb, rowptr, colidx, lu, dinv, w, z);
    for (size_t e = 0; e < n; ++e) x[e] += z[e];
    if (conv) {
      status = 0;
      break;
    }
    if (k >= maxit) {
      status = 1;
      break;
    }
    orc_spmv(nb, rowptr, colidx, vals, x, w);
    for (size_t e = 0; e < n; ++e) r[e] = b[e] - w[e];
    beta = sqrt(dot(n, r, r));
    if (beta <= tol) {
      status = 0;
      break;
    }
  }
stop:
  *iters = k;
done:
  if (status == -6) {
    *relres = NAN;
  } else if (n0 == 0.0) {
    *relres = 0.0;
  } else {
    orc_spmv(nb, rowptr, colidx, vals, x, w);
    double nres = 0.0;
    for (size_t e = 0; e < n; ++e) nres += (b[e] - w[e]) * (b[e] - w[e]);
    *relres = sqrt(nres) / n0;
  }
  free(V); free(w); free(z); free(r); free(H); free(cs); free(sn); free(g); free(y); free(h1); free(h2);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting, A x = b in place      */
/* (brute-force reference for tiny systems).  a is n x n row-major.         */
/* Returns 0 or -1 when singular.                                           */
/* ------------------------------------------------------------------------ */
int orc_dense_solve(int32_t n, double *a, double *b) {
  for (int32_t col = 0; col < n; ++col) {
    int32_t piv = col;
    for (int32_t r = col + 1; r < n; ++r)
      if (fabs(a[(size_t)r * n + col]) > fabs(a[(size_t)piv * n + col])) piv = r;
    if (a[(size_t)piv * n + col] == 0.0) return -1;
    if (piv != col) {
      for (int32_t c = 0; c < n; ++c) {
        double t = a[(size_t)col * n + c];
        a[(size_t)col * n + c] = a[(size_t)piv * n + c];
        a[(size_t)piv * n + c] = t;
      }
      double t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
    for (int32_t r = col + 1; r < n; ++r) {
      double f = a[(size_t)r * n + col] / a[(size_t)col * n + col];
      if (f == 0.0) continue;
      for (int32_t c = col; c < n; ++c) a[(size_t)r * n + c] -= f * a[(size_t)col * n + c];
      b[r] -= f * b[col];
    }
  }
  for (int32_t r = n - 1; r >= 0; --r) {
    double acc = b[r];
    for (int32_t c = r + 1; c < n; ++c) acc -= a[(size_t)r * n + c] * b[c];
    b[r] = acc / a[(size_t)r * n + r];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Parallel schedules (Section 4.4).  Both work on the symmetrised pattern  */
/* (an edge i-j whenever block (i,j) or (j,i) is present).                  */
/*                                                                          */
/* Level scheduling: level(i) = 0 if i has no neighbour j < i, else         */
/* 1 + max level(j) over its neighbours j < i.  Rows of one level have no   */
/* edge between them, every edge joins rows of different levels, and        */
/* ordering rows by level keeps every edge's direction, so the ILU0 of the  */
/* level-ordered matrix is the natural-order ILU0 relabelled.               */
/*                                                                          */
/* Graph colouring: greedy first fit in natural row order, each row taking  */
/* the smallest colour not used by a neighbour coloured before it.          */
/*                                                                          */
/* Both return the number of sets; key[i] is the set of row i.  The        */
/* adjacency is built here from the pattern (CSR of the symmetrised graph). */
/* ------------------------------------------------------------------------ */
static void sym_graph(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int64_t **gptr,
                      int32_t **gadj) {
  int64_t *deg = calloc((size_t)nb + 1, sizeof(int64_t));
  for (int32_t i = 0; i < nb; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j == i) continue;
      deg[i]++;
      deg[j]++;
    }
  int64_t *ptr = calloc((size_t)nb + 1, sizeof(int64_t));
  for (int32_t i = 0; i < nb; ++i) ptr[i + 1] = ptr[i] + deg[i];
  int32_t *adj = malloc(sizeof(int32_t) * (size_t)(ptr[nb] ? ptr[nb] : 1));
  int64_t *fill = calloc((size_t)nb, sizeof(int64_t));
  for (int32_t i = 0; i < nb; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j == i) continue;
      adj[ptr[i] + fill[i]++] = j;
      adj[ptr[j] + fill[j]++] = i;
    }
  free(deg);
  free(fill);
  *gptr = ptr;
  *gadj = adj;
}

int32_t orc_levels(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int32_t *level) {
  int64_t *gptr;
  int32_t *gadj;
  sym_graph(nb, rowptr, colidx, &gptr, &gadj);
  int32_t nlev = 0;
  for (int32_t i = 0; i < nb; ++i) {
    int32_t l = 0;
    for (int64_t m = gptr[i]; m < gptr[i + 1]; ++m) {
      int32_t j = gadj[m];
      if (j < i && level[j] + 1 > l) l = level[j] + 1;
    }
    level[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  free(gptr);
  free(gadj);
  return nlev;
}

int32_t orc_colours(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int32_t *colour) {
  int64_t *gptr;
  int32_t *gadj;
  sym_graph(nb, rowptr, colidx, &gptr, &gadj);
  int32_t ncol = 0;
  for (int32_t i = 0; i < nb; ++i) colour[i] = -1;
  for (int32_t i = 0; i < nb; ++i) {
    int32_t c = 0;
    for (;;) { /* smallest colour unused by an already coloured neighbour */
      int used = 0;
      for (int64_t m = gptr[i]; m < gptr[i + 1]; ++m)
        if (colour[gadj[m]] == c) {
          used = 1;
          break;
        }
      if (!used) break;
      ++c;
    }
    colour[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(gptr);
  free(gadj);
  return ncol;
}

/*
 * Sub-key that orders the rows of each set (level or colour, Section 4.4):
 * out[i] = 2 key[i] + open[i], where row i is open when some neighbour in
 * the symmetrised pattern lies in a later set.  Rows of one set share no
 * edge, so any order inside a set gives the same factors up to the order of
 * each row's sums; closed rows (no later neighbour, hence no U block) first.
 */
void orc_closed_first_key(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const int32_t *key,
                          int32_t *out) {
  for (int32_t i = 0; i < nb; ++i) out[i] = 2 * key[i];
  for (int32_t i = 0; i < nb; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (key[j] > key[i]) out[i] = 2 * key[i] + 1;
      if (key[i] > key[j]) out[j] = 2 * key[j] + 1;
    }
}

/* binary min-heap of int64 keys (smallest-last colouring below) */
typedef struct {
  int64_t *k;
  int64_t n, cap;
} orc_heap;

static void heap_push(orc_heap *h, int64_t key) {
  if (h->n == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 1024;
    h->k = realloc(h->k, sizeof(int64_t) * (size_t)h->cap);
  }
  int64_t i = h->n++;
  while (i > 0 && h->k[(i - 1) / 2] > key) {
    h->k[i] = h->k[(i - 1) / 2];
    i = (i - 1) / 2;
  }
  h->k[i] = key;
}

static int64_t heap_pop(orc_heap *h) {
  int64_t top = h->k[0], last = h->k[--h->n], i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= h->n) break;
    if (c + 1 < h->n && h->k[c + 1] < h->k[c]) ++c;
    if (h->k[c] >= last) break;
    h->k[i] = h->k[c];
    i = c;
  }
  if (h->n > 0) h->k[i] = last;
  return top;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/*
 * Greedy colouring in smallest-last order (Matula & Beck 1983, one of the
 * colouring reorders Section 4.4 leaves open): the rows are removed one at a
 * time from the symmetrised pattern, each time a row of least degree
 * (distinct neighbours still present; ties to the lowest row), and then
 * coloured first-fit in the reverse order of removal.  Returns the number
 * of colours.
 */
/* The symmetrised pattern with each row's distinct neighbours sorted
   (no self loops): row i's neighbours are gadj[dptr[i] .. dptr[i+1]). */
static void distinct_graph(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int64_t **dptr_out,
                           int32_t **gadj_out) {
  int64_t *gptr;
  int32_t *gadj;
  sym_graph(nb, rowptr, colidx, &gptr, &gadj);
  int64_t *dptr = malloc(sizeof(int64_t) * ((size_t)nb + 1));
  int64_t w = 0;
  dptr[0] = 0;
  for (int32_t i = 0; i < nb; ++i) {
    int64_t a = gptr[i], b = gptr[i + 1];
    qsort(gadj + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
    for (int64_t m = a; m < b; ++m)
      if (m == a || gadj[m] != gadj[m - 1]) gadj[w++] = gadj[m];
    dptr[i + 1] = w;
  }
  free(gptr);
  *dptr_out = dptr;
  *gadj_out = gadj;
}

static int32_t colours_sl_graph(int32_t nb, const int64_t *dptr, const int32_t *gadj, int32_t *colour);

int32_t orc_colours_sl(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int32_t *colour) {
  int64_t *dptr;
  int32_t *gadj;
  distinct_graph(nb, rowptr, colidx, &dptr, &gadj);
  int32_t ncol = colours_sl_graph(nb, dptr, gadj, colour);
  free(dptr);
  free(gadj);
  return ncol;
}

static int32_t colours_sl_graph(int32_t nb, const int64_t *dptr, const int32_t *gadj, int32_t *colour) {
  int32_t *deg = malloc(sizeof(int32_t) * (size_t)(nb ? nb : 1));
  char *gone = calloc((size_t)(nb ? nb : 1), 1);
  int32_t *order = malloc(sizeof(int32_t) * (size_t)(nb ? nb : 1));
  orc_heap h = {0, 0, 0};
  for (int32_t i = 0; i < nb; ++i) {
    deg[i] = (int32_t)(dptr[i + 1] - dptr[i]);
    heap_push(&h, ((int64_t)deg[i] << 32) | (int64_t)i);
  }
  int32_t cnt = 0;
  while (h.n > 0) {
    int64_t key = heap_pop(&h);
    int32_t v = (int32_t)(key & 0xffffffff), d = (int32_t)(key >> 32);
    if (gone[v] || d != deg[v]) continue; /* a stale entry */
    gone[v] = 1;
    order[cnt++] = v;
    for (int64_t m = dptr[v]; m < dptr[v + 1]; ++m) {
      int32_t u = gadj[m];
      if (!gone[u]) {
        deg[u]--;
        heap_push(&h, ((int64_t)deg[u] << 32) | (int64_t)u);
      }
    }
  }
  int32_t ncol = 0;
  int32_t *stamp = malloc(sizeof(int32_t) * ((size_t)nb + 1));
  for (int32_t i = 0; i <= nb; ++i) stamp[i] = -1;
  for (int32_t i = 0; i < nb; ++i) colour[i] = -1;
  for (int32_t t = cnt - 1; t >= 0; --t) {
    int32_t v = order[t];
    for (int64_t m = dptr[v]; m < dptr[v + 1]; ++m)
      if (colour[gadj[m]] >= 0) stamp[colour[gadj[m]]] = v;
    int32_t c = 0;
    while (stamp[c] == v) ++c;
    colour[v] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(h.k);
  free(stamp);
  free(order);
  free(gone);
  free(deg);
  return ncol;
}

/*
 * Colour-class reduction by Kempe chains (Kempe 1879) after the
 * smallest-last colouring: the highest class is emptied row by row if it
 * can be, then the next, until a class cannot be emptied or two colours
 * remain.  A row v of the highest colour t first takes the smallest colour
 * below t that none of its neighbours has.  Otherwise, for each pair of
 * colours (a, b) below t (a ascending, then b ascending, b != a), the rows
 * reachable from v's a-coloured neighbours through rows coloured a or b
 * (breadth first: the starts in neighbour order, then each row's
 * neighbours in order) are collected; if the search meets no neighbour of
 * v and stays within kempe_cap rows, a and b are exchanged on the
 * collected rows (a proper colouring stays proper, and no neighbour of v
 * keeps colour a) and v takes a.  A row that finds no such pair keeps t.
 * Returns the number of colours.
 */
enum { kempe_cap = 16384 };

int32_t orc_colours_kempe(int32_t nb, const int32_t *rowptr, const int32_t *colidx, int32_t *colour) {
  int64_t *dptr;
  int32_t *gadj;
  distinct_graph(nb, rowptr, colidx, &dptr, &gadj);
  int32_t ncol = colours_sl_graph(nb, dptr, gadj, colour);
  int32_t *nbr_of = malloc(sizeof(int32_t) * (size_t)(nb ? nb : 1)); /* row whose neighbour this is */
  int32_t *mark = malloc(sizeof(int32_t) * (size_t)(nb ? nb : 1));   /* search that collected it */
  int32_t *queue = malloc(sizeof(int32_t) * (size_t)(kempe_cap + 1));
  int32_t *used = calloc((size_t)ncol + 1, sizeof(int32_t));
  for (int32_t i = 0; i < nb; ++i) nbr_of[i] = mark[i] = -1;
  int32_t search = 0;
  while (ncol > 2) {
    const int32_t t = ncol - 1;
    int32_t left = 0;
    for (int32_t v = 0; v < nb; ++v) {
      if (colour[v] != t) continue;
      for (int32_t c = 0; c < t; ++c) used[c] = 0;
      for (int64_t m = dptr[v]; m < dptr[v + 1]; ++m) {
        nbr_of[gadj[m]] = v;
        if (colour[gadj[m]] < t) used[colour[gadj[m]]] = 1;
      }
      int32_t free_c = -1;
      for (int32_t c = 0; c < t && free_c < 0; ++c)
        if (!used[c]) free_c = c;
      if (free_c >= 0) {
        colour[v] = free_c;
        continue;
      }
      int done = 0;
      for (int32_t a = 0; a < t && !done; ++a)
        for (int32_t b = 0; b < t && !done; ++b) {
          if (b == a) continue;
          ++search;
          int32_t qn = 0, ok = 1;
          for (int64_t m = dptr[v]; m < dptr[v + 1] && ok; ++m) {
            const int32_t u = gadj[m];
            if (colour[u] != a) continue;
            if (qn == kempe_cap) ok = 0;
            else {
              mark[u] = search;
              queue[qn++] = u;
            }
          }
          for (int32_t head = 0; head < qn && ok; ++head) {
            const int32_t x = queue[head];
            for (int64_t m = dptr[x]; m < dptr[x + 1]; ++m) {
              const int32_t y = gadj[m];
              if (mark[y] == search || (colour[y] != a && colour[y] != b)) continue;
              if (nbr_of[y] == v || qn == kempe_cap) {
                ok = 0;
                break;
              }
              mark[y] = search;
              queue[qn++] = y;
            }
          }
          if (ok) {
            for (int32_t q = 0; q < qn; ++q) colour[queue[q]] = colour[queue[q]] == a ? b : a;
            colour[v] = a;
            done = 1;
          }
        }
      if (!done) ++left;
    }
    if (left > 0) break;
    --ncol;
  }
  free(used);
  free(queue);
  free(mark);
  free(nbr_of);
  free(dptr);
  free(gadj);
  return ncol;
}

/* perm[new] = old: rows ordered by key, natural order inside each key
   (a stable counting sort) */
void orc_order_by_key(int32_t nb, const int32_t *key, int32_t nkeys, int32_t *perm) {
  int64_t *start = calloc((size_t)nkeys + 1, sizeof(int64_t));
  for (int32_t i = 0; i < nb; ++i) start[key[i] + 1]++;
  for (int32_t k = 0; k < nkeys; ++k) start[k + 1] += start[k];
  for (int32_t i = 0; i < nb; ++i) perm[start[key[i]]++] = i;
  free(start);
}

/*
 * P A P^T for perm[new] = old: new row i' is old row perm[i'], its columns
 * renumbered by the inverse permutation and sorted.  Output arrays are
 * sized like the input (prowptr nb+1, pcolidx nnzb, pvals 9*nnzb).
 */
void orc_permute(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                 const int32_t *perm, int32_t *prowptr, int32_t *pcolidx, double *pvals) {
  int32_t *iperm = malloc(sizeof(int32_t) * (size_t)nb);
  for (int32_t i = 0; i < nb; ++i) iperm[perm[i]] = i;
  prowptr[0] = 0;
  for (int32_t ni = 0; ni < nb; ++ni) {
    int32_t oi = perm[ni];
    int64_t len = rowptr[oi + 1] - rowptr[oi];
    int64_t base = prowptr[ni];
    prowptr[ni + 1] = (int32_t)(base + len);
    /* insertion sort of the renumbered columns, carrying the blocks along */
    for (int64_t q = 0; q < len; ++q) {
      int64_t m = rowptr[oi] + q;
      int32_t nc = iperm[colidx[m]];
      int64_t at = base + q;
      while (at > base && pcolidx[at - 1] > nc) {
        pcolidx[at] = pcolidx[at - 1];
        memcpy(pvals + BS2 * at, pvals + BS2 * (at - 1), sizeof(double) * BS2);
        --at;
      }
      pcolidx[at] = nc;
      memcpy(pvals + BS2 * at, vals + BS2 * m, sizeof(double) * BS2);
    }
  }
  free(iperm);
}
