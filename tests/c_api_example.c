/* A C program that uses the library through include/did.h only: no Python,
 * no PyTorch.  It factorises a small planted matrix given on the command line
 * as M N K sweeps, with X written by the program itself (host memory), runs
 * the sweeps, reads the factors back and prints one line:
 *   ok <iters> <f(B,C)> <trace first> <trace last> <min B> <min C>
 * and on any error "error <status> <message>" with a non-zero exit code.
 * X[m + j*M] = sum_{k < K+2} (1 + (m + k) % 7) / 7 * (1 + (j + 2k) % 5) / 5,
 * nonnegative and of rank above K (no exact fit); the start point is the
 * library's seeded one. */
#include <stdio.h>
#include <stdlib.h>

#include "did.h"

int main(int argc, char** argv) {
  if (argc < 5) {
    fprintf(stderr, "usage: %s M N K sweeps\n", argv[0]);
    return 2;
  }
  const int64_t M = atoll(argv[1]), N = atoll(argv[2]);
  const int32_t K = atoi(argv[3]), sweeps = atoi(argv[4]);
  float* X = (float*)malloc(sizeof(float) * (size_t)(M * N));
  float* B = (float*)malloc(sizeof(float) * (size_t)(M * K));
  float* C = (float*)malloc(sizeof(float) * (size_t)(K * N));
  double* trace = (double*)malloc(sizeof(double) * (size_t)(sweeps + 1));
  if (!X || !B || !C || !trace) return 3;
  for (int64_t j = 0; j < N; ++j)
    for (int64_t m = 0; m < M; ++m) {
      double v = 0.0;
      for (int k = 0; k < K + 2; ++k) v += (1.0 + (double)((m + k) % 7)) / 7.0 * (1.0 + (double)((j + 2 * k) % 5)) / 5.0;
      X[m + j * M] = (float)v;
    }

  did_options o;
  did_default_options(&o);
  o.refresh_every = 4;
  did_ctx* ctx = NULL;
  did_status st = did_create_ex(X, M, N, K, 11, &o, &ctx);
  if (st != DID_OK) {
    printf("error %d %s\n", (int)st, did_status_string(st));
    return 1;
  }
  st = did_sweep(ctx, sweeps);
  double f = 0.0;
  if (st == DID_OK) st = did_objective(ctx, &f);
  if (st == DID_OK) st = did_get_factors(ctx, B, C);
  int32_t n = 0;
  if (st == DID_OK) st = did_get_trace(ctx, trace, sweeps + 1, &n);
  if (st != DID_OK) {
    printf("error %d %s\n", (int)st, did_last_error(ctx));
    did_destroy(ctx);
    return 1;
  }
  float bmin = B[0], cmin = C[0];
  for (int64_t i = 0; i < M * K; ++i) bmin = B[i] < bmin ? B[i] : bmin;
  for (int64_t i = 0; i < K * N; ++i) cmin = C[i] < cmin ? C[i] : cmin;
  printf("ok %d %.17g %.17g %.17g %g %g\n", (int)n - 1, f, trace[0], trace[n - 1], (double)bmin, (double)cmin);
  did_destroy(ctx);
  free(X);
  free(B);
  free(C);
  free(trace);
  return 0;
}
