/* A plain C caller of the library: the C-ABI of include/bicoptor.h used
 * without Python.  Shares plaintexts, runs the ReLU (Alg. relu) and the fused
 * product -> truncation -> ReLU step on host buffers, reconstructs, and checks
 * the results against the plaintext.  Prints "ok" and exits 0 on success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "bicoptor.h"

#define N 4099
#define FAIL(...) do { fprintf(stderr, __VA_ARGS__); return 1; } while (0)

int main(void) {
  bc_ctx *ctx = NULL;
  int rc = bc_create(&ctx, 0xC0FFEEull, 0, NULL);
  if (rc) FAIL("bc_create: %s\n", bc_strerror(rc));

  /* plaintexts: integers in (-2^20, 2^20), fixed point with f = 16 bits */
  int64_t *x = malloc(N * sizeof(int64_t)), *y = malloc(N * sizeof(int64_t));
  for (int i = 0; i < N; ++i) {
    x[i] = ((int64_t)((i * 2654435761u) % 2000000u) - 1000000) ;
    y[i] = (int64_t)((i % 7) + 1) << 16;           /* 1..7 in fixed point */
  }

  /* device ReLU */
  int64_t *dx, *dy, *rec;
  uint64_t *s0, *s1, *r0, *r1;
  if (cudaMalloc((void **)&dx, N * 8) || cudaMalloc((void **)&dy, N * 8) ||
      cudaMalloc((void **)&rec, N * 8) || cudaMalloc((void **)&s0, N * 8) ||
      cudaMalloc((void **)&s1, N * 8) || cudaMalloc((void **)&r0, N * 8) ||
      cudaMalloc((void **)&r1, N * 8))
    FAIL("cudaMalloc\n");
  cudaMemcpy(dx, x, N * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dy, y, N * 8, cudaMemcpyHostToDevice);
  bc_drelu_params prm = {64, 24, 0, 0};
  if ((rc = bc_share(ctx, 64, dx, N, 1, s0, s1))) FAIL("bc_share: %s\n", bc_strerror(rc));
  if ((rc = bc_relu(ctx, &prm, s0, s1, N, 2, r0, r1))) FAIL("bc_relu: %s\n", bc_strerror(rc));
  if ((rc = bc_reconstruct(ctx, 64, r0, r1, N, rec))) FAIL("bc_reconstruct: %s\n", bc_strerror(rc));
  if ((rc = bc_synchronize(ctx))) FAIL("bc_synchronize: %s\n", bc_strerror(rc));
  int64_t *h = malloc(N * sizeof(int64_t));
  cudaMemcpy(h, rec, N * 8, cudaMemcpyDeviceToHost);
  for (int i = 0; i < N; ++i)
    if (h[i] != (x[i] > 0 ? x[i] : 0)) FAIL("relu mismatch at %d: %lld vs %lld\n", i,
                                            (long long)h[i], (long long)x[i]);

  /* the fused step on pinned host buffers: ReLU(trunc_16(x * y)) = ReLU(x * y / 2^16) +- 1 */
  uint64_t *hx0, *hx1, *hy0, *hy1, *hr0, *hr1;
  cudaMallocHost((void **)&hx0, N * 8); cudaMallocHost((void **)&hx1, N * 8);
  cudaMallocHost((void **)&hy0, N * 8); cudaMallocHost((void **)&hy1, N * 8);
  cudaMallocHost((void **)&hr0, N * 8); cudaMallocHost((void **)&hr1, N * 8);
  uint64_t *t0, *t1;
  if (cudaMalloc((void **)&t0, N * 8) || cudaMalloc((void **)&t1, N * 8)) FAIL("cudaMalloc\n");
  bc_share(ctx, 64, dy, N, 3, t0, t1);
  bc_synchronize(ctx);
  cudaMemcpy(hx0, s0, N * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(hx1, s1, N * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(hy0, t0, N * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(hy1, t1, N * 8, cudaMemcpyDeviceToHost);
  bc_linear_relu_args a = {0};
  a.ring_bits = 64; a.trunc_bits = 16; a.relu = prm;
  a.x0 = hx0; a.x1 = hx1; a.y0 = hy0; a.y1 = hy1; a.n = N; a.tensor_id = 4;
  a.relu0 = hr0; a.relu1 = hr1;
  if ((rc = bc_linear_relu_host(ctx, &a))) FAIL("bc_linear_relu_host: %s\n", bc_strerror(rc));
  for (int i = 0; i < N; ++i) {
    const int64_t got = (int64_t)(hr0[i] + hr1[i]);
    const int64_t want = (x[i] * (y[i] >> 16) > 0) ? x[i] * (y[i] >> 16) : 0;
    if (got - want > 1 || want - got > 1) FAIL("linear relu mismatch at %d: %lld vs %lld\n", i,
                                               (long long)got, (long long)want);
  }
  bc_comm c;
  bc_get_comm(ctx, &c);
  if (c.p0_to_p2 != 2ull * N * 25 * 25) FAIL("comm counter %llu\n", (unsigned long long)c.p0_to_p2);
  bc_destroy(ctx);
  printf("ok\n");
  return 0;
}
