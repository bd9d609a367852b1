// Microbenchmarks of the integer units that bound the hot path (a measuring
// aid; the paper has no counterpart).  Each kernel runs CHAINS independent
// dependency chains per thread of one instruction kind over a full-occupancy
// grid, so the chains' latency is hidden and the pipe's issue rate shows:
//   Philox-4x32 round      two 32 x 32 -> 64 products and two three-input
//                          XORs with round keys from the constant bank, the
//                          form of the hot path's widening products (a
//                          multiply-add chain feeding both halves back runs
//                          slower on GB300, so it would understate the ceiling)
//   low multiply-add       x = x * x + c (32-bit; the square keeps a compiler
//                          from folding unrolled steps into one)
//   logic + add            x = (x ^ c) + K (two integer-ALU instructions)
//   high product           x = hi32(x * K) ^ c (the form of the hot path's
//                          64 x 32 draws and shuffle indices; the XOR goes to
//                          the ALU pipe)
// One CTA also reads its SM's cycle counter against the global nanosecond
// timer, so the rates can be expressed per SM clock.
#include "bc_internal.h"

namespace bc {
namespace {

constexpr int kChains = 8;
__constant__ uint32_t kPeakKeys[8] = {0x9E3779B9u, 0x3C6EF372u, 0xDAA66D2Bu, 0x78DDE6E4u,
                                      0xBB67AE85u, 0x76CF5D0Au, 0x32370B8Fu, 0xED9EBA14u};
constexpr int kPeakCtasPerSm = 8;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int KIND>
__global__ void __launch_bounds__(kBlock)
    int_peak_kernel(uint32_t seed, int iters, uint64_t* __restrict__ sink,
                    unsigned long long* __restrict__ clock_probe) {
  uint32_t a[kChains], b[kChains], c[kChains], d[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    a[j] = seed ^ (threadIdx.x * 0x9E3779B9u + (uint32_t)j * 0x85EBCA6Bu + blockIdx.x);
    b[j] = (uint32_t)j + blockIdx.x;
    c[j] = a[j] * 3u;
    d[j] = b[j] ^ 0x55u;
  }
  const bool probe = blockIdx.x == 0 && threadIdx.x == 0;
  uint64_t c0 = 0, t0 = 0;
  if (probe) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        if (KIND == 0) {          // Philox-4x32 round: two widening products
          const uint64_t p0 = (uint64_t)kPhiloxM0 * a[j];
          const uint64_t p1 = (uint64_t)kPhiloxM1 * c[j];
          const uint32_t n0 = (uint32_t)(p1 >> 32) ^ b[j] ^ kPeakKeys[u];
          const uint32_t n2 = (uint32_t)(p0 >> 32) ^ d[j] ^ kPeakKeys[u + 4];
          b[j] = (uint32_t)p1;
          d[j] = (uint32_t)p0;
          a[j] = n0;
          c[j] = n2;
        } else if (KIND == 1) {   // 32-bit multiply-add
          a[j] = a[j] * a[j] + b[j];
        } else if (KIND == 2) {   // logic + add
          a[j] = (a[j] ^ b[j]) + 0x9E3779B9u;
        } else {                  // high product
          a[j] = __umulhi(a[j], kPeakKeys[u]) ^ b[j];
        }
      }
    }
  }
  if (probe) {
    const uint64_t c1 = clock64();
    const uint64_t t1 = global_ns();
    clock_probe[0] = c1 - c0;
    clock_probe[1] = t1 - t0;
  }
  uint64_t acc = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j)
    acc ^= ((uint64_t)b[j] << 32) ^ a[j] ^ ((uint64_t)c[j] << 17) ^ d[j];
  if (acc == 0x0123456789ABCDEFull) sink[0] = acc;   // keeps every chain live
}

}  // namespace
}  // namespace bc

extern "C" int bc_measure_int_peaks(int device, bc_int_peaks* out) {
  if (!out) return BC_EINVAL;
  *out = bc_int_peaks{};
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return BC_ECUDA;
  int num_sms = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  uint64_t* sink = nullptr;
  unsigned long long* probe = nullptr;
  int rc = BC_OK;
  do {
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&probe, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      rc = BC_ECUDA;
      break;
    }
    const unsigned grid = (unsigned)num_sms * bc::kPeakCtasPerSm;
    const int iters = 16384;
    double* rates[4] = {&out->imad_wide_per_s, &out->imad_per_s, &out->alu_per_s,
                        &out->imad_hi_per_s};
    // instructions of the measured kind per thread: iters x 4 x chains, x2 for the two
    // products of a Philox round and for logic + add
    const double per_thread[4] = {iters * 8.0 * bc::kChains, iters * 4.0 * bc::kChains,
                                  iters * 8.0 * bc::kChains, iters * 4.0 * bc::kChains};
    for (int kind = 0; kind < 4 && rc == BC_OK; ++kind) {
      for (int rep = 0; rep < 3 && rc == BC_OK; ++rep) {   // first run warms the clocks
        cudaEventRecord(e0, s);
        if (kind == 0) bc::int_peak_kernel<0><<<grid, bc::kBlock, 0, s>>>(rep, iters, sink, probe);
        if (kind == 1) bc::int_peak_kernel<1><<<grid, bc::kBlock, 0, s>>>(rep, iters, sink, probe);
        if (kind == 2) bc::int_peak_kernel<2><<<grid, bc::kBlock, 0, s>>>(rep, iters, sink, probe);
        if (kind == 3) bc::int_peak_kernel<3><<<grid, bc::kBlock, 0, s>>>(rep, iters, sink, probe);
        cudaEventRecord(e1, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
          rc = BC_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double r = per_thread[kind] * grid * bc::kBlock / (ms * 1e-3);
        if (r > *rates[kind]) *rates[kind] = r;
        unsigned long long h[2] = {0, 0};
        if (cudaMemcpy(h, probe, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) {
          rc = BC_ECUDA;
          break;
        }
        if (h[1]) out->sm_mhz = 1e3 * (double)h[0] / (double)h[1];
      }
    }
    out->sm_count = num_sms;
    if (cudaGetLastError() != cudaSuccess) rc = BC_ECUDA;
  } while (0);
  cudaFree(sink);
  cudaFree(probe);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return rc;
}
