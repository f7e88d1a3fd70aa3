/* A plain C11 client of mgsa_qr_noalloc across a device reset.  The caller
 * owns (and allocates) its inputs and outputs; the library allocates nothing
 * and keeps its scratch in a static device array whose address, like the
 * kernel's shared-memory limit, belongs to the CUDA context.  This program
 * factors the same A = tridiag(-1, 2.1, -1) and Z twice in the form given on
 * the command line, with cudaDeviceReset (which ends this process's own
 * context) and fresh allocations in between, and checks that the second call
 * still runs (its set-up is redone in the new context) and gives the same R
 * and Q bit for bit.  Prints "ok" and exits 0, or the reason and exits 1.
 * Without a usable GPU it prints "nogpu" and exits 0.
 *
 *   noalloc_reset <m> <n> <variant 0..2> */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "mgsa.h"

static double zval(long k, int j) { return sin(0.29 * (double)(k + 1) * (double)(j + 1)) + 0.02 * (double)j; }

/* One allocation-free QR on freshly allocated device buffers; Q, R to host. */
static int run_once(long m, int n, int v, const int32_t* rowptr, const int32_t* col, const double* val, long nnz,
                    const double* Z, double* Q, double* R) {
  int32_t *d_rp = NULL, *d_col = NULL, *d_info = NULL;
  double *d_val = NULL, *d_Z = NULL, *d_Q = NULL, *d_R = NULL;
  if (cudaMalloc((void**)&d_rp, sizeof(int32_t) * (size_t)(m + 1)) ||
      cudaMalloc((void**)&d_col, sizeof(int32_t) * (size_t)nnz) ||
      cudaMalloc((void**)&d_val, sizeof(double) * (size_t)nnz) ||
      cudaMalloc((void**)&d_Z, sizeof(double) * (size_t)(m * n)) ||
      cudaMalloc((void**)&d_Q, sizeof(double) * (size_t)(m * n)) ||
      cudaMalloc((void**)&d_R, sizeof(double) * (size_t)(n * n)) || cudaMalloc((void**)&d_info, 2 * sizeof(int32_t))) {
    printf("cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(d_rp, rowptr, sizeof(int32_t) * (size_t)(m + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_Z, Z, sizeof(double) * (size_t)(m * n), cudaMemcpyHostToDevice);
  mgsa_csr A = {m, nnz, d_rp, d_col, d_val};
  mgsa_status st = mgsa_qr_noalloc(&A, d_Z, m, n, m, (mgsa_variant)v, d_Q, m, d_R, n, d_info, NULL);
  if (st != MGSA_OK) {
    printf("mgsa_qr_noalloc failed: status %d %s\n", (int)st, mgsa_last_error());
    return 1;
  }
  int32_t info[2] = {-1, -1};
  if (cudaMemcpy(info, d_info, sizeof(info), cudaMemcpyDeviceToHost) != cudaSuccess) {
    printf("copy of info failed\n");
    return 1;
  }
  if (info[0] != 0 || info[1] != 0) {
    printf("QR failed on the device: %d %d\n", info[0], info[1]);
    return 1;
  }
  cudaMemcpy(Q, d_Q, sizeof(double) * (size_t)(m * n), cudaMemcpyDeviceToHost);
  cudaMemcpy(R, d_R, sizeof(double) * (size_t)(n * n), cudaMemcpyDeviceToHost);
  cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val); cudaFree(d_Z); cudaFree(d_Q); cudaFree(d_R); cudaFree(d_info);
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const long m = atol(argv[1]);
  const int n = atoi(argv[2]);
  const int v = atoi(argv[3]);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    printf("nogpu\n");
    return 0;
  }
  const long nnz = 3 * m - 2;
  int32_t* rowptr = malloc(sizeof(int32_t) * (size_t)(m + 1));
  int32_t* col = malloc(sizeof(int32_t) * (size_t)nnz);
  double* val = malloc(sizeof(double) * (size_t)nnz);
  double* Z = malloc(sizeof(double) * (size_t)(m * n));
  double* Q1 = malloc(sizeof(double) * (size_t)(m * n));
  double* Q2 = malloc(sizeof(double) * (size_t)(m * n));
  double* R1 = malloc(sizeof(double) * (size_t)(n * n));
  double* R2 = malloc(sizeof(double) * (size_t)(n * n));
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

  if (run_once(m, n, v, rowptr, col, val, nnz, Z, Q1, R1)) return 1;
  if (cudaDeviceReset() != cudaSuccess) {
    printf("cudaDeviceReset failed\n");
    return 1;
  }
  if (run_once(m, n, v, rowptr, col, val, nnz, Z, Q2, R2)) return 1;
  if (memcmp(R1, R2, sizeof(double) * (size_t)(n * n)) != 0 || memcmp(Q1, Q2, sizeof(double) * (size_t)(m * n)) != 0) {
    printf("results differ after the reset\n");
    return 1;
  }
  for (int j = 0; j < n; ++j)
    if (!(R1[j + j * n] > 0.0)) { printf("diag %d not positive\n", j); return 1; }
  printf("ok %.17g\n", R1[0]);
  free(rowptr); free(col); free(val); free(Z); free(Q1); free(Q2); free(R1); free(R2);
  return 0;
}
