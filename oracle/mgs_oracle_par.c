/*
 * Multi-core build of the CPU oracle's row-oriented algorithms
 * (Imakura & Yamamoto, arXiv 1703.10440, Algorithms 4, 7 and 8).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes: exactly what oracle_mgs(variant, form = row) of
 * mgs_oracle.c computes, operation for operation and bit for bit, with the
 * independent loops spread over OpenMP threads:
 *   - every CSR row of a matrix-vector product (and of the block product
 *     X = A Z of Algorithm 8) is one task, summed in ascending nonzero order;
 *   - the element-wise scalings q_i = z_i / r_ii, p_i = x_i / r_ii are split
 *     over rows;
 *   - at step i, each column j > i is one task: r_ij = p_i^T z_j (ascending
 *     dot), z_j <- z_j - r_ij q_i and (Algorithm 8) x_j <- x_j - r_ij p_i.
 *     Every column sees the same operations in the same order as in the
 *     single-thread loop, since the columns are independent within a step;
 *   - the one reduction that spans rows, s = z_i^T x_i, stays a single
 *     ascending sum on one thread.
 * So the result does not depend on the number of threads, and equals the
 * single-thread oracle's bitwise (a CPU test checks this).  Compiled with
 * -ffp-contract=off like the single-thread oracle; without OpenMP the pragmas
 * are ignored and it runs on one thread.
 *
 * Storage and breakdown convention as in mgs_oracle.c: Z, Q column-major
 * (ldz, ldq >= m), R column-major n x n (ldr >= n) with zeros below the
 * diagonal; returns 0 or the 1-based breakdown column j (*kind = 1 for
 * z_j^T x_j <= 0, 2 for NaN/Inf); -1 for invalid arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the parallel loops use (1 when built without OpenMP). */
int oracle_par_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set the thread count of later calls (ignored without OpenMP). */
void oracle_par_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* y = A x, one task per row, each row summed in ascending nonzero order. */
static void par_csr_mv(int64_t m, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                       double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/* a^T b, ascending, on the calling thread. */
static double seq_dot(int64_t m, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t k = 0; k < m; ++k) s += a[k] * b[k];
  return s;
}

/* y = x / alpha, split over rows. */
static void par_scale_div(int64_t m, const double* x, double alpha, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < m; ++k) y[k] = x[k] / alpha;
}

static int diag_verdict(double s, int* kind) {
  if (s != s || s == INFINITY || s == -INFINITY) { *kind = 2; return 0; }
  if (!(s > 0.0)) { *kind = 1; return 0; }
  return 1;
}

/* Right-looking MGS in the form `variant` (0 naive = Algorithm 4, 1 HA =
 * Algorithm 7, 2 HP = Algorithm 8). */
int oracle_par_mgs_row(int variant, int64_t m, int n, const int32_t* rowptr, const int32_t* col, const double* val,
                       const double* Z, int64_t ldz, double* Q, int64_t ldq, double* R, int ldr, int* kind) {
  if (variant < 0 || variant > 2 || n < 1 || m < n || ldz < m || ldq < m || ldr < n) return -1;
  const int hp = variant == 2;
  /* naive: x (A z_i) and p (A q_i); HA: x and p; HP: X (m x n, x_j then p_j) */
  double* X = (double*)malloc(sizeof(double) * (size_t)m * (size_t)(hp ? n : 2));
  if (!X) return -1;
  int info = 0;
  *kind = 0;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) R[i + (int64_t)j * ldr] = 0.0;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) memcpy(Q + (int64_t)j * ldq, Z + (int64_t)j * ldz, (size_t)m * sizeof(double));
  if (hp) {
    /* X = A Z, the block product: every (row, column) entry one ascending sum. */
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r)
      for (int j = 0; j < n; ++j) {
        const double* zj = Q + (int64_t)j * ldq;
        double s = 0.0;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) s += val[e] * zj[col[e]];
        X[r + (int64_t)j * m] = s;
      }
  }
  for (int i = 0; i < n; ++i) {
    double* zi = Q + (int64_t)i * ldq;
    double* xi = hp ? X + (int64_t)i * m : X;  /* x_i */
    double* pi = hp ? xi : X + m;               /* p_i (HP: in place of x_i) */
    if (!hp) par_csr_mv(m, rowptr, col, val, zi, xi); /* x_i = A z_i^{(i-1)} */
    const double s = seq_dot(m, zi, xi);              /* r_ii^2 = z_i^T x_i */
    if (!diag_verdict(s, kind)) { info = i + 1; break; }
    const double rii = sqrt(s);
    R[i + (int64_t)i * ldr] = rii;
    par_scale_div(m, zi, rii, zi); /* q_i = z_i / r_ii */
    if (variant == 0) par_csr_mv(m, rowptr, col, val, zi, pi); /* p_i = A q_i */
    else par_scale_div(m, xi, rii, pi);                         /* p_i = x_i / r_ii (eq. (tec1)) */
    /* Row i of R and the rank-1 updates, one column per task. */
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = i + 1; j < n; ++j) {
      double* zj = Q + (int64_t)j * ldq;
      const double rij = seq_dot(m, pi, zj); /* r_ij = p_i^T z_j^{(i-1)} */
      R[i + (int64_t)j * ldr] = rij;
      for (int64_t k = 0; k < m; ++k) zj[k] = zj[k] - rij * zi[k]; /* z_j^{(i)} */
      if (hp) {
        double* xj = X + (int64_t)j * m;
        for (int64_t k = 0; k < m; ++k) xj[k] = xj[k] - rij * pi[k]; /* x_j^{(i)} (eq. (tec2)) */
      }
    }
  }
  free(X);
  return info;
}
