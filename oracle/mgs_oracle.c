/*
 * CPU oracle for the A-inner-product modified Gram-Schmidt thin QR
 * (Imakura & Yamamoto, "Efficient implementations of the modified
 * Gram-Schmidt orthogonalization with a non-standard inner product",
 * arXiv 1703.10440).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Section 1, eq. (1)): for Z (m x n, m >= n) and a sparse
 * symmetric positive definite A (m x m, CSR), the factors Q (m x n) and R
 * (n x n, upper triangular, positive diagonal) with Z = QR and Q^T A Q = I_n.
 *
 * Six algorithms, each written out in the order and notation of the paper:
 *   Algorithm 3  MGS-naive(col)   2n matrix-vector products (MV)
 *   Algorithm 4  MGS-naive(row)   2n MV
 *   Algorithm 5  MGS-HA(col)      n MV, p_j = x_j / r_jj  (eq. (tec1))
 *   Algorithm 7  MGS-HA(row)      n MV
 *   Algorithm 6  MGS-HP(col)      one block product X = AZ, x-recurrence (eq. (tec2))
 *   Algorithm 8  MGS-HP(row)      one block product X = AZ
 * and the classical Gram-Schmidt counterparts CGS-naive / CGS-HA / CGS-HP in
 * both forms (Section 2.3 and Section 3.3: the same recurrences with
 * r_ij = p_i^T z_j^{(0)}, i.e. every coefficient of column j taken against the
 * original column instead of the partly orthogonalised one).
 *
 * Arithmetic conventions (the paper fixes none of these):
 *   - IEEE binary64 throughout; the file is compiled with -ffp-contract=off,
 *     so every a*b+c rounds twice exactly as written;
 *   - every dot product and every CSR row sum runs in ascending index order;
 *   - q = z / r and p = x / r are true divisions, element by element;
 *   - Algorithm 6's  x_j^{(j-1)} = x_j^{(0)} - sum_{i<j} r_ij p_i  is evaluated
 *     left to right, one subtraction per i in ascending order; that is the
 *     same operation sequence as Algorithm 8's per-step update
 *     x_j <- x_j - r_ij p_i, which is how the garbled x line of Algorithm 8 is
 *     read (at the end of step i, every j > i is updated with p_i).
 *   - Breakdown (the paper assumes full column rank, Section 1): when
 *     z_j^T x_j is not > 0 the routine stops and returns j (1-based); *kind is
 *     1 for a non-positive value and 2 for NaN/Inf.  Columns >= j of Q and R
 *     are left as they are.
 *
 * Storage: Z, Q column-major with leading dimensions ldz, ldq >= m; R
 * column-major n x n with leading dimension ldr >= n, written in full with
 * zeros below the diagonal.  Q may not alias Z.
 *
 * The metric helpers at the end evaluate ||Z - QR||_F, ||I - Q^T A Q||_F and
 * the Cholesky factor of Z^T A Z in double-double or long double arithmetic.
 */
#include <math.h>
#include <stdint.h>

/* ORACLE_MUTANT (test builds only) plants one known mistake so that the test
 * suite can show its pins catch it:
 *   1  MGS-HA forms p_j = A q_j with a second MV (i.e. it becomes naive)
 *   2  MGS-HP leaves x_j = A z_j^{(0)} (drops eq. (tec2)'s recurrence)
 *   3  the rank-1 update adds instead of subtracting
 *   4  r_ij uses the Euclidean inner product q_i^T z_j instead of p_i^T z_j
 *   5  CGS takes r_ij against the working z_j^{(i-1)} (i.e. it becomes MGS)
 * The default build (ORACLE_MUTANT undefined or 0) has none of them. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#include <stdlib.h>
#include <string.h>

#define OR_OK 0

/* ---------------------------------------------------------------------- */
/* Basic kernels (Section 3, eqs. (error_AXPY)-(error_MV) name these ops) */
/* ---------------------------------------------------------------------- */

/* y = A x for CSR A, each row summed in ascending nonzero order. */
static void csr_mv(int64_t m, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* x, double* y) {
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/* a^T b, ascending. */
static double dot(int64_t m, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t k = 0; k < m; ++k) s += a[k] * b[k];
  return s;
}

/* y = y - alpha * x  (the AXPY of eq. (AXPY)). */
static void axpy_sub(int64_t m, double alpha, const double* x, double* y) {
#if ORACLE_MUTANT == 3
  for (int64_t k = 0; k < m; ++k) y[k] = y[k] + alpha * x[k];
#else
  for (int64_t k = 0; k < m; ++k) y[k] = y[k] - alpha * x[k];
#endif
}

/* y = x / alpha  (the scaling of eq. (scaling)). */
static void scale_div(int64_t m, const double* x, double alpha, double* y) {
  for (int64_t k = 0; k < m; ++k) y[k] = x[k] / alpha;
}

/* r_jj = sqrt(s) with the breakdown rule stated in the header. */
static int diag_ok(double s, int* kind) {
  if (s != s || s == INFINITY || s == -INFINITY) { *kind = 2; return 0; }
  if (!(s > 0.0)) { *kind = 1; return 0; }
  return 1;
}

static void copy_cols(int64_t m, int n, const double* Z, int64_t ldz, double* Q, int64_t ldq) {
  for (int j = 0; j < n; ++j) memcpy(Q + (int64_t)j * ldq, Z + (int64_t)j * ldz, (size_t)m * sizeof(double));
}

static void zero_R(int n, double* R, int ldr) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) R[i + (int64_t)j * ldr] = 0.0;
}

#define QC(j) (Q + (int64_t)(j) * ldq)
#define RR(i, j) R[(i) + (int64_t)(j) * ldr]

/* ---------------------------------------------------------------------- */
/* Algorithm 3: MGS-naive(col).  2n MV.                                    */
/* Working storage: Q's column j holds z_j^{(i)} until it becomes q_j.     */
/* ---------------------------------------------------------------------- */
int oracle_mgs_naive_col(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                         int64_t* mv_count, int* kind) {
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n); /* p_i = A q_i */
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  for (int j = 0; j < n && !info; ++j) {
    double* zj = QC(j);
    for (int i = 0; i < j; ++i) {
      RR(i, j) = dot(m, P + (int64_t)i * m, zj); /* r_ij = p_i^T z_j^{(i-1)} */
      axpy_sub(m, RR(i, j), QC(i), zj);          /* z_j^{(i)} = z_j^{(i-1)} - r_ij q_i */
    }
    csr_mv(m, rowptr, col, val, zj, x); /* x_j^{(j-1)} = A z_j^{(j-1)} */
    ++*mv_count;
    double s = dot(m, zj, x);
    if (!diag_ok(s, kind)) { info = j + 1; break; }
    RR(j, j) = sqrt(s);                           /* r_jj = sqrt(z^T x) */
    scale_div(m, zj, RR(j, j), zj);               /* q_j = z_j^{(j-1)} / r_jj */
    csr_mv(m, rowptr, col, val, zj, P + (int64_t)j * m); /* p_j = A q_j */
    ++*mv_count;
  }
  free(P);
  free(x);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 4: MGS-naive(row).  2n MV.  Same operations as Algorithm 3    */
/* in right-looking order (Section 2.1 says the two agree exactly).         */
/* ---------------------------------------------------------------------- */
int oracle_mgs_naive_row(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                         int64_t* mv_count, int* kind) {
  double* p = (double*)malloc(sizeof(double) * (size_t)m);
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  for (int i = 0; i < n; ++i) {
    double* zi = QC(i);
    csr_mv(m, rowptr, col, val, zi, x); /* x_i^{(i-1)} = A z_i^{(i-1)} */
    ++*mv_count;
    double s = dot(m, zi, x);
    if (!diag_ok(s, kind)) { info = i + 1; break; }
    RR(i, i) = sqrt(s);
    scale_div(m, zi, RR(i, i), zi);      /* q_i */
    csr_mv(m, rowptr, col, val, zi, p); /* p_i = A q_i */
    ++*mv_count;
    for (int j = i + 1; j < n; ++j) {
#if ORACLE_MUTANT == 4
      RR(i, j) = dot(m, zi, QC(j));
#else
      RR(i, j) = dot(m, p, QC(j));   /* r_ij = p_i^T z_j^{(i-1)} */
#endif
      axpy_sub(m, RR(i, j), zi, QC(j)); /* z_j^{(i)} */
    }
  }
  free(p);
  free(x);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 5: MGS-HA(col).  n MV; p_j = x_j^{(j-1)} / r_jj (eq. (tec1)). */
/* ---------------------------------------------------------------------- */
int oracle_mgs_ha_col(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                      int64_t* mv_count, int* kind) {
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  for (int j = 0; j < n && !info; ++j) {
    double* zj = QC(j);
    for (int i = 0; i < j; ++i) {
      RR(i, j) = dot(m, P + (int64_t)i * m, zj);
      axpy_sub(m, RR(i, j), QC(i), zj);
    }
    csr_mv(m, rowptr, col, val, zj, x); /* x_j^{(j-1)} = A z_j^{(j-1)} */
    ++*mv_count;
    double s = dot(m, zj, x);
    if (!diag_ok(s, kind)) { info = j + 1; break; }
    RR(j, j) = sqrt(s);
    scale_div(m, zj, RR(j, j), zj);                 /* q_j = z_j / r_jj */
    scale_div(m, x, RR(j, j), P + (int64_t)j * m);  /* p_j = x_j / r_jj */
  }
  free(P);
  free(x);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 7: MGS-HA(row).  n MV.                                        */
/* ---------------------------------------------------------------------- */
int oracle_mgs_ha_row(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                      int64_t* mv_count, int* kind) {
  double* p = (double*)malloc(sizeof(double) * (size_t)m);
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  for (int i = 0; i < n; ++i) {
    double* zi = QC(i);
    csr_mv(m, rowptr, col, val, zi, x); /* x_i^{(i-1)} = A z_i^{(i-1)} */
    ++*mv_count;
    double s = dot(m, zi, x);
    if (!diag_ok(s, kind)) { info = i + 1; break; }
    RR(i, i) = sqrt(s);
    scale_div(m, zi, RR(i, i), zi); /* q_i */
#if ORACLE_MUTANT == 1
    csr_mv(m, rowptr, col, val, zi, p);
#else
    scale_div(m, x, RR(i, i), p);   /* p_i = x_i / r_ii */
#endif
    for (int j = i + 1; j < n; ++j) {
#if ORACLE_MUTANT == 4
      RR(i, j) = dot(m, zi, QC(j));
#else
      RR(i, j) = dot(m, p, QC(j));
#endif
      axpy_sub(m, RR(i, j), zi, QC(j));
    }
  }
  free(p);
  free(x);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 6: MGS-HP(col).  X = AZ as one block product; the A-images are */
/* carried by the recurrence of eq. (tec2).                                 */
/* ---------------------------------------------------------------------- */
int oracle_mgs_hp_col(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                      int64_t* mv_count, int* kind) {
  double* X = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n); /* column j: x_j, then p_j */
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  /* X = [x_1^{(0)}, ..., x_n^{(0)}] = A Z : one block product of n columns. */
  for (int j = 0; j < n; ++j) csr_mv(m, rowptr, col, val, QC(j), X + (int64_t)j * m);
  *mv_count = 1;
  for (int j = 0; j < n && !info; ++j) {
    double* zj = QC(j);
    double* xj = X + (int64_t)j * m;
    for (int i = 0; i < j; ++i) {
      RR(i, j) = dot(m, X + (int64_t)i * m, zj); /* r_ij = p_i^T z_j^{(i-1)} */
      axpy_sub(m, RR(i, j), QC(i), zj);
    }
    /* x_j^{(j-1)} = x_j^{(0)} - sum_{i<j} r_ij p_i, ascending i. */
    for (int i = 0; i < j; ++i) axpy_sub(m, RR(i, j), X + (int64_t)i * m, xj);
    double s = dot(m, zj, xj);
    if (!diag_ok(s, kind)) { info = j + 1; break; }
    RR(j, j) = sqrt(s);
    scale_div(m, zj, RR(j, j), zj); /* q_j */
    scale_div(m, xj, RR(j, j), xj); /* p_j = x_j^{(j-1)} / r_jj */
  }
  free(X);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 8: MGS-HP(row).  X = AZ once; at the end of step i every      */
/* x_j (j > i) is updated with p_i.                                         */
/* ---------------------------------------------------------------------- */
int oracle_mgs_hp_row(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
                      int64_t* mv_count, int* kind) {
  double* X = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  for (int j = 0; j < n; ++j) csr_mv(m, rowptr, col, val, QC(j), X + (int64_t)j * m);
  *mv_count = 1;
  for (int i = 0; i < n; ++i) {
    double* zi = QC(i);
    double* xi = X + (int64_t)i * m;
    double s = dot(m, zi, xi); /* r_ii = sqrt(z_i^T x_i) */
    if (!diag_ok(s, kind)) { info = i + 1; break; }
    RR(i, i) = sqrt(s);
    scale_div(m, zi, RR(i, i), zi); /* q_i */
    scale_div(m, xi, RR(i, i), xi); /* p_i */
    for (int j = i + 1; j < n; ++j) {
#if ORACLE_MUTANT == 4
      RR(i, j) = dot(m, zi, QC(j));
#else
      RR(i, j) = dot(m, xi, QC(j));
#endif
      axpy_sub(m, RR(i, j), zi, QC(j));
    }
#if ORACLE_MUTANT != 2
    for (int j = i + 1; j < n; ++j) axpy_sub(m, RR(i, j), xi, X + (int64_t)j * m); /* x_j^{(i)} */
#endif
  }
  free(X);
  return info;
}

/* ---------------------------------------------------------------------- */
/* Successive orthogonalisation (Section 2.1: the column-oriented MGS is   */
/* the one suited to it).  Given k columns Qo (m x k) that are already     */
/* A-orthonormal and Po (= A Qo as the algorithm produced it), the n new    */
/* columns Z are A-orthonormalised against them and among themselves by     */
/* continuing Algorithm 3 (naive), 5 (HA) or 6 (HP) at column k+1.         */
/* Outputs: Q (m x n), P (m x n, the p_j of the new columns), R ((k+n) x n, */
/* column-major, ldr >= k+n: rows 0..k-1 hold r_ij against the old columns, */
/* rows k..k+n-1 the new upper triangle).  With k = 0 this is Algorithm     */
/* 3 / 5 / 6 itself, and appending to the result of the first k columns     */
/* performs exactly the operations of one run over all k + n columns.      */
/* ---------------------------------------------------------------------- */
int oracle_mgs_append(int variant, int64_t m, int k, int n, const int32_t* rowptr, const int32_t* col,
                      const double* val, const double* Qo, int64_t ldqo, const double* Po, int64_t ldpo,
                      const double* Z, int64_t ldz, double* Q, int64_t ldq, double* P, int64_t ldp, double* R,
                      int ldr, int64_t* mv_count, int* kind) {
  if (m < 1 || n < 1 || k < 0 || m < k + n || ldz < m || ldq < m || ldp < m || ldr < k + n) return -1;
  if (k > 0 && (!Qo || !Po || ldqo < m || ldpo < m)) return -1;
  double* X = (variant == 2) ? (double*)malloc(sizeof(double) * (size_t)m * (size_t)n) : NULL;
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < k + n; ++i) R[i + (int64_t)j * ldr] = 0.0;
  copy_cols(m, n, Z, ldz, Q, ldq);
  if (variant == 2) {
    for (int j = 0; j < n; ++j) csr_mv(m, rowptr, col, val, QC(j), X + (int64_t)j * m); /* X = A Z */
    *mv_count = 1;
  }
  for (int j = 0; j < n && !info; ++j) {
    double* zj = QC(j);
    /* r_ij and z_j^{(i)} against the old columns, then the new ones (ascending i) */
    for (int i = 0; i < k; ++i) {
      R[i + (int64_t)j * ldr] = dot(m, Po + (int64_t)i * ldpo, zj);
      axpy_sub(m, R[i + (int64_t)j * ldr], Qo + (int64_t)i * ldqo, zj);
    }
    for (int i = 0; i < j; ++i) {
      R[k + i + (int64_t)j * ldr] = dot(m, P + (int64_t)i * ldp, zj);
      axpy_sub(m, R[k + i + (int64_t)j * ldr], QC(i), zj);
    }
    const double* xj;
    if (variant == 2) {
      double* xw = X + (int64_t)j * m; /* x_j^{(j-1)} = x_j^{(0)} - sum_i r_ij p_i (eq. (tec2)) */
      for (int i = 0; i < k; ++i) axpy_sub(m, R[i + (int64_t)j * ldr], Po + (int64_t)i * ldpo, xw);
      for (int i = 0; i < j; ++i) axpy_sub(m, R[k + i + (int64_t)j * ldr], P + (int64_t)i * ldp, xw);
      xj = xw;
    } else {
      csr_mv(m, rowptr, col, val, zj, x); /* x_j^{(j-1)} = A z_j^{(j-1)} */
      ++*mv_count;
      xj = x;
    }
    double s = dot(m, zj, xj);
    if (!diag_ok(s, kind)) { info = j + 1; break; }
    const double r = sqrt(s);
    R[k + j + (int64_t)j * ldr] = r;
    scale_div(m, zj, r, zj); /* q_j */
    if (variant == 0) {
      csr_mv(m, rowptr, col, val, zj, P + (int64_t)j * ldp); /* p_j = A q_j */
      ++*mv_count;
    } else {
      scale_div(m, xj, r, P + (int64_t)j * ldp); /* p_j = x_j / r_jj (eq. (tec1)) */
    }
  }
  free(X);
  free(x);
  return info;
}

/* ---------------------------------------------------------------------- */
/* CGS (Section 2.3; Section 3.3 states the recurrences): Algorithms 3/5/6 */
/* and 4/7/8 with r_ij = p_i^T z_j^{(0)}.  Q's column j holds the working  */
/* z_j^{(i)}; Z's column j keeps z_j^{(0)}.                                 */
/* ---------------------------------------------------------------------- */

/* r_ij of CGS: against the original column z0 (mutant 5: the working one). */
static double cgs_coef(int64_t m, const double* p, const double* z0, const double* zwork) {
#if ORACLE_MUTANT == 5
  (void)z0;
  return dot(m, p, zwork);
#else
  (void)zwork;
  return dot(m, p, z0);
#endif
}

/* Column form: for each j, r_ij (i < j) and z_j^{(i)} in ascending i, then
 * x_j (naive / HA: one MV; HP: x_j^{(0)} - sum_i r_ij p_i), r_jj, q_j and p_j
 * (naive: A q_j; HA / HP: x_j / r_jj, eq. (tec1)). */
int oracle_cgs_col(int variant, int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr, int64_t* mv_count,
                   int* kind) {
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n); /* HP: x_j, then p_j */
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  if (variant == 2) {
    for (int j = 0; j < n; ++j) csr_mv(m, rowptr, col, val, QC(j), P + (int64_t)j * m); /* X = A Z */
    *mv_count = 1;
  }
  for (int j = 0; j < n && !info; ++j) {
    double* zj = QC(j);
    const double* z0 = Z + (int64_t)j * ldz;
    for (int i = 0; i < j; ++i) {
      RR(i, j) = cgs_coef(m, P + (int64_t)i * m, z0, zj); /* r_ij = p_i^T z_j^{(0)} */
      axpy_sub(m, RR(i, j), QC(i), zj);                   /* z_j^{(i)} = z_j^{(i-1)} - r_ij q_i */
    }
    double* xj;
    if (variant == 2) {
      xj = P + (int64_t)j * m; /* x_j^{(j-1)} = x_j^{(0)} - sum_{i<j} r_ij p_i, ascending i */
      for (int i = 0; i < j; ++i) axpy_sub(m, RR(i, j), P + (int64_t)i * m, xj);
    } else {
      csr_mv(m, rowptr, col, val, zj, x); /* x_j^{(j-1)} = A z_j^{(j-1)} */
      ++*mv_count;
      xj = x;
    }
    double s = dot(m, zj, xj);
    if (!diag_ok(s, kind)) { info = j + 1; break; }
    RR(j, j) = sqrt(s);
    scale_div(m, zj, RR(j, j), zj); /* q_j */
    if (variant == 0) {
      csr_mv(m, rowptr, col, val, zj, P + (int64_t)j * m); /* p_j = A q_j */
      ++*mv_count;
    } else {
      scale_div(m, xj, RR(j, j), P + (int64_t)j * m); /* p_j = x_j / r_jj */
    }
  }
  free(P);
  free(x);
  return info;
}

/* Row form: at step i, q_i and p_i, then r_ij = p_i^T z_j^{(0)} and
 * z_j^{(i)} (HP also x_j^{(i)}) for every j > i.  Same operations on every
 * column as the column form, in the same order, hence the same results. */
int oracle_cgs_row(int variant, int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr, int64_t* mv_count,
                   int* kind) {
  double* X = (variant == 2) ? (double*)malloc(sizeof(double) * (size_t)m * (size_t)n) : NULL;
  double* p = (double*)malloc(sizeof(double) * (size_t)m);
  double* x = (double*)malloc(sizeof(double) * (size_t)m);
  int info = 0;
  *kind = 0;
  *mv_count = 0;
  zero_R(n, R, ldr);
  copy_cols(m, n, Z, ldz, Q, ldq);
  if (variant == 2) {
    for (int j = 0; j < n; ++j) csr_mv(m, rowptr, col, val, QC(j), X + (int64_t)j * m);
    *mv_count = 1;
  }
  for (int i = 0; i < n; ++i) {
    double* zi = QC(i);
    double* xi;
    if (variant == 2) {
      xi = X + (int64_t)i * m;
    } else {
      csr_mv(m, rowptr, col, val, zi, x); /* x_i^{(i-1)} = A z_i^{(i-1)} */
      ++*mv_count;
      xi = x;
    }
    double s = dot(m, zi, xi);
    if (!diag_ok(s, kind)) { info = i + 1; break; }
    RR(i, i) = sqrt(s);
    scale_div(m, zi, RR(i, i), zi); /* q_i */
    if (variant == 0) {
      csr_mv(m, rowptr, col, val, zi, p); /* p_i = A q_i */
      ++*mv_count;
    } else {
      scale_div(m, xi, RR(i, i), p); /* p_i = x_i / r_ii */
    }
    for (int j = i + 1; j < n; ++j) {
      RR(i, j) = cgs_coef(m, p, Z + (int64_t)j * ldz, QC(j)); /* r_ij = p_i^T z_j^{(0)} */
      axpy_sub(m, RR(i, j), zi, QC(j));
    }
    if (variant == 2)
      for (int j = i + 1; j < n; ++j) axpy_sub(m, RR(i, j), p, X + (int64_t)j * m); /* x_j^{(i)} */
  }
  free(X);
  free(p);
  free(x);
  return info;
}

/* Dispatcher: variant 0 = naive, 1 = HA, 2 = HP; form 0 = col, 1 = row. */
int oracle_mgs(int variant, int form, int64_t m, int n, const int32_t* rowptr, const int32_t* col,
               const double* val, const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
               int64_t* mv_count, int* kind) {
  if (m < 1 || n < 1 || m < n || ldz < m || ldq < m || ldr < n) return -1;
  switch (variant * 2 + form) {
    case 0: return oracle_mgs_naive_col(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    case 1: return oracle_mgs_naive_row(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    case 2: return oracle_mgs_ha_col(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    case 3: return oracle_mgs_ha_row(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    case 4: return oracle_mgs_hp_col(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    case 5: return oracle_mgs_hp_row(m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
    default: return -1;
  }
}

/* CGS dispatcher, same conventions as oracle_mgs. */
int oracle_cgs(int variant, int form, int64_t m, int n, const int32_t* rowptr, const int32_t* col,
               const double* val, const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr,
               int64_t* mv_count, int* kind) {
  if (m < 1 || n < 1 || m < n || ldz < m || ldq < m || ldr < n) return -1;
  if (variant < 0 || variant > 2 || form < 0 || form > 1) return -1;
  return form == 0 ? oracle_cgs_col(variant, m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind)
                   : oracle_cgs_row(variant, m, n, rowptr, col, val, Z, ldz, Q, ldq, R, ldr, mv_count, kind);
}

/* y = A x in FP64, exported for tests of the generators. */
void oracle_csr_mv(int64_t m, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                   double* y) {
  csr_mv(m, rowptr, col, val, x, y);
}

/* ---------------------------------------------------------------------- */
/* Metrics in double-double arithmetic (error-free transforms:             */
/* Knuth's TwoSum and Dekker's TwoProduct with Veltkamp splitting, so that  */
/* no fused multiply-add is needed).                                        */
/* ---------------------------------------------------------------------- */
typedef struct { double hi, lo; } dd;

static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *s = x;
  *e = (a - av) + (b - bv);
}

static void split(double a, double* hi, double* lo) {
  const double c = 134217729.0; /* 2^27 + 1 */
  double t = c * a;
  double h = t - (t - a);
  *hi = h;
  *lo = a - h;
}

static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  double ah, al, bh, bl;
  split(a, &ah, &al);
  split(b, &bh, &bl);
  *p = x;
  *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
}

static dd dd_add_d(dd a, double b) {
  double s, e;
  two_sum(a.hi, b, &s, &e);
  e += a.lo;
  double hi, lo;
  two_sum(s, e, &hi, &lo);
  dd r = {hi, lo};
  return r;
}

static dd dd_add(dd a, dd b) {
  double s, e;
  two_sum(a.hi, b.hi, &s, &e);
  e += a.lo + b.lo;
  double hi, lo;
  two_sum(s, e, &hi, &lo);
  dd r = {hi, lo};
  return r;
}

static dd dd_fma_dd(dd acc, double a, double b) { /* acc + a*b, product exact */
  double p, e;
  two_prod(a, b, &p, &e);
  dd t = {p, e};
  return dd_add(acc, t);
}

/* ||Z - QR||_F and ||Z||_F, each entry (Z - QR)_kj accumulated in double-double. */
void oracle_repr_error(int64_t m, int n, const double* Z, int64_t ldz, const double* Q, int64_t ldq,
                       const double* R, int ldr, double* err_f, double* z_f) {
  dd e2 = {0.0, 0.0}, z2 = {0.0, 0.0};
  for (int j = 0; j < n; ++j) {
    for (int64_t k = 0; k < m; ++k) {
      dd acc = {Z[k + (int64_t)j * ldz], 0.0};
      for (int i = 0; i <= j; ++i) acc = dd_fma_dd(acc, -Q[k + (int64_t)i * ldq], R[i + (int64_t)j * ldr]);
      double d = acc.hi + acc.lo;
      e2 = dd_fma_dd(e2, d, d);
      double zz = Z[k + (int64_t)j * ldz];
      z2 = dd_fma_dd(z2, zz, zz);
    }
  }
  *err_f = sqrt(e2.hi + e2.lo);
  *z_f = sqrt(z2.hi + z2.lo);
}

/* G = Q^T A Q in double-double (A Q by exact products, double-double sums);
 * returns ||I - G||_F and writes G (n x n, column-major) if G != NULL. */
double oracle_orth_loss(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const double* Q, int64_t ldq, double* G) {
  dd* AQ = (dd*)malloc(sizeof(dd) * (size_t)m * (size_t)n);
  for (int j = 0; j < n; ++j) {
    const double* qj = Q + (int64_t)j * ldq;
    for (int64_t r = 0; r < m; ++r) {
      dd s = {0.0, 0.0};
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) s = dd_fma_dd(s, val[e], qj[col[e]]);
      AQ[r + (int64_t)j * m] = s;
    }
  }
  dd f2 = {0.0, 0.0};
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      const double* qi = Q + (int64_t)i * ldq;
      dd s = {0.0, 0.0};
      for (int64_t k = 0; k < m; ++k) {
        dd a = AQ[k + (int64_t)j * m];
        s = dd_fma_dd(s, qi[k], a.hi);
        s = dd_fma_dd(s, qi[k], a.lo);
      }
      if (G) G[i + (int64_t)j * n] = s.hi + s.lo;
      dd d = dd_add_d(s, i == j ? -1.0 : 0.0);
      double dv = d.hi + d.lo;
      f2 = dd_fma_dd(f2, dv, dv);
    }
  }
  free(AQ);
  return sqrt(f2.hi + f2.lo);
}

/* Upper Cholesky factor of Z^T A Z computed in long double (tiny inputs only:
 * long double is software binary128 on some hosts).  Returns 0, or k+1 if the
 * Gram matrix is not positive definite at pivot k. */
int oracle_chol_gram_ld(int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const double* Z, int64_t ldz, double* Rout, int ldr) {
  long double* AZ = (long double*)malloc(sizeof(long double) * (size_t)m * (size_t)n);
  long double* G = (long double*)malloc(sizeof(long double) * (size_t)n * (size_t)n);
  for (int j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      long double s = 0.0L;
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
        s += (long double)val[e] * (long double)Z[col[e] + (int64_t)j * ldz];
      AZ[r + (int64_t)j * m] = s;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      long double s = 0.0L;
      for (int64_t k = 0; k < m; ++k) s += (long double)Z[k + (int64_t)i * ldz] * AZ[k + (int64_t)j * m];
      G[i + (int64_t)j * n] = s;
    }
  /* symmetrise (exact arithmetic makes G symmetric) */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < j; ++i) {
      long double a = 0.5L * (G[i + (int64_t)j * n] + G[j + (int64_t)i * n]);
      G[i + (int64_t)j * n] = a;
      G[j + (int64_t)i * n] = a;
    }
  int info = 0;
  long double* U = (long double*)calloc((size_t)n * (size_t)n, sizeof(long double));
  for (int j = 0; j < n && !info; ++j) {
    long double d = G[j + (int64_t)j * n];
    for (int k = 0; k < j; ++k) d -= U[k + (int64_t)j * n] * U[k + (int64_t)j * n];
    if (!(d > 0.0L)) { info = j + 1; break; }
    U[j + (int64_t)j * n] = sqrtl(d);
    for (int i = j + 1; i < n; ++i) {
      long double s = G[j + (int64_t)i * n];
      for (int k = 0; k < j; ++k) s -= U[k + (int64_t)j * n] * U[k + (int64_t)i * n];
      U[j + (int64_t)i * n] = s / U[j + (int64_t)j * n];
    }
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) Rout[i + (int64_t)j * ldr] = (double)U[i + (int64_t)j * n];
  free(U);
  free(G);
  free(AZ);
  return info;
}
