/* A plain C caller of the library's C ABI (include/spmv_gb300.h), no Python or PyTorch:
 * the 5-point Laplacian (4 on the diagonal, -1 to each grid neighbour) on an n x n grid
 * applied to u(i, j) = i^2 + j^2. Every value is an integer below 2^53, so each row sum is
 * exact in any order: interior rows give -4, boundary rows 4 u - (sum of the neighbours
 * inside the grid). Runs the profile route, a device-buffer run, a host-buffer run and the
 * error paths; prints "ok" and exits 0 on success. */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>

#include "spmv_gb300.h"

#define N_GRID 200

static int fail(const char *what, int code) {
  fprintf(stderr, "FAIL %s (%d)\n", what, code);
  return 1;
}

static double u_of(long i, long j) { return (double)(i * i + j * j); }

int main(void) {
  const long n = N_GRID, N = n * n;
  int32_t *rowptr = malloc(sizeof(int32_t) * (size_t)(N + 1));
  int32_t *colind = malloc(sizeof(int32_t) * (size_t)(5 * N));
  double *val = malloc(sizeof(double) * (size_t)(5 * N));
  double *x = malloc(sizeof(double) * (size_t)N);
  double *y = malloc(sizeof(double) * (size_t)N);
  double *want = malloc(sizeof(double) * (size_t)N);
  if (!rowptr || !colind || !val || !x || !y || !want) return fail("host allocation", 0);
  long k = 0;
  for (long r = 0; r < N; ++r) {
    const long i = r % n, j = r / n;
    rowptr[r] = (int32_t)k;
    double w = 4.0 * u_of(i, j);
    /* columns in increasing order: (i, j-1), (i-1, j), (i, j), (i+1, j), (i, j+1) */
    if (j > 0) { colind[k] = (int32_t)(r - n); val[k++] = -1.0; w -= u_of(i, j - 1); }
    if (i > 0) { colind[k] = (int32_t)(r - 1); val[k++] = -1.0; w -= u_of(i - 1, j); }
    colind[k] = (int32_t)r;
    val[k++] = 4.0;
    if (i < n - 1) { colind[k] = (int32_t)(r + 1); val[k++] = -1.0; w -= u_of(i + 1, j); }
    if (j < n - 1) { colind[k] = (int32_t)(r + n); val[k++] = -1.0; w -= u_of(i, j + 1); }
    x[r] = u_of(i, j);
    want[r] = w;
  }
  rowptr[N] = (int32_t)k;
  const int64_t nnz = k;

  spmv_handle_t h = NULL;
  int st = spmv_create(&h, N, N, nnz, rowptr, colind, val, SPMV_F64, 0, NULL);
  if (st != SPMV_OK) return fail(spmv_status_string((spmv_status)st), st);

  double *dx = NULL, *dy = NULL;
  if (cudaMalloc((void **)&dx, sizeof(double) * (size_t)N) != cudaSuccess ||
      cudaMalloc((void **)&dy, sizeof(double) * (size_t)N) != cudaSuccess)
    return fail("cudaMalloc", 0);
  if (cudaMemcpy(dx, x, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail("upload x", 0);

  st = spmv_run(h, dx, dy, NULL);   /* no variant installed yet */
  if (st != SPMV_ERR_NOT_TUNED) return fail("run before tune", st);

  spmv_tune_report rep;
  st = spmv_tune(h, SPMV_TUNE_PROFILE, NULL, &rep, NULL);
  if (st != SPMV_OK) return fail("spmv_tune", st);
  st = spmv_run(h, dx, dy, NULL);
  if (st != SPMV_OK) return fail("spmv_run", st);
  if (cudaMemcpy(y, dy, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail("download y", 0);
  for (long r = 0; r < N; ++r)
    if (y[r] != want[r]) return fail("device-buffer y differs from the closed form", (int)r);

  for (long r = 0; r < N; ++r) y[r] = -1.0;
  st = spmv_run_host(h, x, y, NULL);
  if (st != SPMV_OK) return fail("spmv_run_host", st);
  for (long r = 0; r < N; ++r)
    if (y[r] != want[r]) return fail("host-buffer y differs from the closed form", (int)r);

  if (spmv_run(h, NULL, dy, NULL) != SPMV_ERR_ARG) return fail("null x accepted", 0);
  int32_t code = -1;
  if (spmv_get_last_device_error(h, &code) != SPMV_OK || code != 0)
    return fail("device error word", code);
  if (spmv_destroy(h) != SPMV_OK) return fail("spmv_destroy", 0);
  cudaFree(dx);
  cudaFree(dy);
  free(rowptr); free(colind); free(val); free(x); free(y); free(want);
  printf("ok classes=%u variant=(%d,%d,%d,%d,%d)\n", rep.classes, rep.variant.partition,
         rep.variant.index, rep.variant.xpath, rep.variant.vec, rep.variant.vs);
  return 0;
}
