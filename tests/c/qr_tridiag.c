/* A plain C11 client of libmgsa: no C++, no Python.  Builds A = tridiag(-1,
 * 2.1, -1) (m x m, CSR) and Z (m x n, deterministic values), runs mgsa_qr in
 * the form given on the command line through the C ABI, and checks on the
 * host that R is upper triangular with a positive diagonal, that
 * ||Z - QR||_F / ||Z||_F and ||I - Q^T A Q||_F are small.  Prints one line
 * "ok <repr> <loss> <r_00> <r_11>" and exits 0, or prints the reason and
 * exits 1.  Without a usable GPU it prints "nogpu <status>" and exits 0
 * (mgsa_create must fail cleanly).
 *
 *   qr_tridiag <m> <n> <variant 0..5> [R output file] */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "mgsa.h"

static double zval(long k, int j) { return sin(0.37 * (double)(k + 1) * (double)(j + 1)) + 0.01 * (double)j; }

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const long m = atol(argv[1]);
  const int n = atoi(argv[2]);
  const int v = atoi(argv[3]);
  mgsa_handle h = NULL;
  mgsa_status st = mgsa_create(&h, 0);
  if (st != MGSA_OK) {
    printf("nogpu %d %s\n", (int)st, mgsa_last_error());
    return 0;
  }
  const long nnz = 3 * m - 2;
  int32_t* rowptr = malloc(sizeof(int32_t) * (size_t)(m + 1));
  int32_t* col = malloc(sizeof(int32_t) * (size_t)nnz);
  double* val = malloc(sizeof(double) * (size_t)nnz);
  double* Z = malloc(sizeof(double) * (size_t)(m * n));
  double* Q = malloc(sizeof(double) * (size_t)(m * n));
  double* R = malloc(sizeof(double) * (size_t)(n * n));
  long e = 0;
  for (long k = 0; k < m; ++k) {
    rowptr[k] = (int32_t)e;
    if (k > 0) { col[e] = (int32_t)(k - 1); val[e++] = -1.0; }
    col[e] = (int32_t)k; val[e++] = 2.1;
    if (k + 1 < m) { col[e] = (int32_t)(k + 1); val[e++] = -1.0; }
  }
  rowptr[m] = (int32_t)e;
  for (int j = 0; j < n; ++j)
    for (long k = 0; k < m; ++k) Z[k + j * m] = zval(k, j);

  int32_t *d_rp, *d_col;
  double *d_val, *d_Z, *d_Q, *d_R;
  if (cudaMalloc((void**)&d_rp, sizeof(int32_t) * (size_t)(m + 1)) || cudaMalloc((void**)&d_col, sizeof(int32_t) * (size_t)nnz) ||
      cudaMalloc((void**)&d_val, sizeof(double) * (size_t)nnz) || cudaMalloc((void**)&d_Z, sizeof(double) * (size_t)(m * n)) ||
      cudaMalloc((void**)&d_Q, sizeof(double) * (size_t)(m * n)) || cudaMalloc((void**)&d_R, sizeof(double) * (size_t)(n * n))) {
    printf("cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(d_rp, rowptr, sizeof(int32_t) * (size_t)(m + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_Z, Z, sizeof(double) * (size_t)(m * n), cudaMemcpyHostToDevice);
  mgsa_csr A = {m, nnz, d_rp, d_col, d_val};
  st = mgsa_qr(h, &A, d_Z, m, n, m, (mgsa_variant)v, d_Q, m, d_R, n, NULL);
  int info = -1;
  if (st == MGSA_OK) st = mgsa_get_info(h, NULL, &info);
  if (st != MGSA_OK || info != 0) {
    printf("mgsa_qr failed: status %d info %d %s\n", (int)st, info, mgsa_last_error());
    return 1;
  }
  cudaMemcpy(Q, d_Q, sizeof(double) * (size_t)(m * n), cudaMemcpyDeviceToHost);
  cudaMemcpy(R, d_R, sizeof(double) * (size_t)(n * n), cudaMemcpyDeviceToHost);

  /* R upper triangular, positive diagonal */
  for (int j = 0; j < n; ++j) {
    if (!(R[j + j * n] > 0.0)) { printf("diag %d not positive\n", j); return 1; }
    for (int i = j + 1; i < n; ++i)
      if (R[i + j * n] != 0.0) { printf("R not upper triangular\n"); return 1; }
  }
  /* ||Z - QR||_F / ||Z||_F */
  double num = 0.0, den = 0.0;
  for (int j = 0; j < n; ++j)
    for (long k = 0; k < m; ++k) {
      double s = 0.0;
      for (int i = 0; i <= j; ++i) s += Q[k + i * m] * R[i + j * n];
      const double d = Z[k + j * m] - s;
      num += d * d;
      den += Z[k + j * m] * Z[k + j * m];
    }
  const double repr = sqrt(num / den);
  /* ||I - Q^T A Q||_F */
  double* AQ = malloc(sizeof(double) * (size_t)(m * n));
  for (int j = 0; j < n; ++j)
    for (long k = 0; k < m; ++k) {
      double s = 0.0;
      for (long p = rowptr[k]; p < rowptr[k + 1]; ++p) s += val[p] * Q[col[p] + j * m];
      AQ[k + j * m] = s;
    }
  double loss = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (long k = 0; k < m; ++k) s += Q[k + i * m] * AQ[k + j * m];
      const double d = (i == j ? 1.0 : 0.0) - s;
      loss += d * d;
    }
  loss = sqrt(loss);
  if (argc > 4) {
    FILE* f = fopen(argv[4], "w");
    if (!f) return 1;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) fprintf(f, "%.17g\n", R[i + j * n]);
    fclose(f);
  }
  printf("ok %.3e %.3e %.17g %.17g\n", repr, loss, R[0], n > 1 ? R[1 + n] : 0.0);
  mgsa_destroy(h);
  cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val); cudaFree(d_Z); cudaFree(d_Q); cudaFree(d_R);
  free(rowptr); free(col); free(val); free(Z); free(Q); free(R); free(AQ);
  return (repr < 1e-13 && loss < 1e-11) ? 0 : 1;
}
