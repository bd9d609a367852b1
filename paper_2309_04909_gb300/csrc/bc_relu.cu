// Fused Bicoptor 2.0 DReLU / ReLU kernels (Alg. drelu, Alg. relu): one tensor
// per launch, the fused product -> truncations -> ReLU step of a linear layer,
// and the RSS variant (Alg. drelu2).  The per-element protocol body is in
// bc_element.cuh; the batched kernels are in bc_batch.cu.
#include "bc_element.cuh"

// The minimum resident CTAs per SM requested from the register allocator for
// the l = 64, lx = 24 single-tensor and fused-step kernels (compile-time; 0 =
// let it choose).  With the slot loop unrolled whole the allocator takes 48
// registers (5 CTAs of 256 threads); six CTAs keep those kernels at 40
// registers without spilling.  Other instantiations (audit buffers, other key
// widths or rings) would spill under the same bound and are left free.
#ifndef BC_RELU_MIN_CTAS
#define BC_RELU_MIN_CTAS 6
#endif

namespace bc {
namespace {

template <typename Lane, int LX, bool SHORT, bool AUDIT>
constexpr int relu_min_ctas() {
  return (sizeof(Lane) == 8 && LX == 24 && SHORT && !AUDIT) ? BC_RELU_MIN_CTAS : 0;
}

// One element per thread; the grid covers the tensor once, so the CTA
// scheduler hands out work as CTAs retire (no static tail).
template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT>
__global__ void __launch_bounds__(kBlock, (relu_min_ctas<Lane, LX, SHORT, AUDIT>()))
    relu_kernel(const ReluConsts k, const Lane* __restrict__ sh0, const Lane* __restrict__ sh1,
                uint64_t n, Lane* __restrict__ o0, Lane* __restrict__ o1, const AuditPtrs aud) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  __shared__ uint64_t r2_s[kMaxSlots];
  uint32_t* perm = perm_s + threadIdx.x;
  if (threadIdx.x < kMaxSlots) r2_s[threadIdx.x] = round2_product(k.tensor_id, threadIdx.x, k.rk);
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  Lane r0, r1;
  bicoptor_element<Lane, LX, SHORT, RELU, AUDIT>(k, k.rk, k.tensor_id, sh0[i], sh1[i],
                                                 k.elem_base + i, perm, r0, r1, aud, i, r2_s);
  o0[i] = r0;
  o1[i] = r1;
}

// Small batches: four lanes per element.  A launch of fewer elements than one
// wave of the one-element-per-thread kernel takes the time of one thread's
// whole key-bit loop (about 27 us at lx = 24), so here the four lanes of an
// element share its work: each expands part of the shuffle stream, lane 0
// applies the shuffle, each lane takes every fourth message slot, the lanes
// OR their zero tests, and the finish's Philox blocks are drawn by different
// lanes.  Same arithmetic and draws as bicoptor_element, so the outputs are
// bit-identical.
constexpr int kSplit = 4;
constexpr int kSplitElems = kBlock / kSplit;   // elements per CTA

template <typename Lane, int LX, bool SHORT, bool RELU>
__global__ void __launch_bounds__(kBlock)
    relu_split_kernel(const ReluConsts k, const Lane* __restrict__ sh0,
                      const Lane* __restrict__ sh1, uint64_t n, Lane* __restrict__ o0,
                      Lane* __restrict__ o1) {
  constexpr uint32_t kSlotsMax = LX ? LX + 1 : kMaxSlots;
  constexpr uint32_t kWordsMax = (kSlotsMax + 3) / 4 * 4;
  __shared__ uint32_t perm_s[kSlotsMax * kSplitElems];
  __shared__ uint32_t words_s[kWordsMax * kSplitElems];
  const uint32_t el = threadIdx.x / kSplit, part = threadIdx.x % kSplit;
  const uint32_t base = (threadIdx.x & 31u) & ~(uint32_t)(kSplit - 1);   // lane of part 0
  const uint64_t i0 = (uint64_t)blockIdx.x * kSplitElems + el;
  const bool valid = i0 < n;
  const uint64_t i = valid ? i0 : n - 1;   // lanes past the end shadow the last element
  const uint32_t lx = LX ? (uint32_t)LX : k.lx;
  const uint32_t L = lx + 1;
  const Lane mask = (Lane)k.ring_mask;
  const RoundKeys& rk = k.rk;
  const ElemPhilox ep(k.elem_base + i, k.tensor_id);
  uint32_t* perm = perm_s + el;
  uint32_t* words = words_s + el;

  // seed01 shuffle stream (steps 1 and 6): block b drawn by lane b mod 4
  const uint32_t nblk = (L + 3) >> 2;
  const StreamPhilox perm_stream(ep, kPair01, kPurPerm, rk);
  for (uint32_t b = part; b < nblk; b += kSplit) {
    const U32x4 wb = perm_stream.block((uint64_t)kPhiloxM1 * b, rk);
    words[(4 * b + 0) * kSplitElems] = wb.x;
    words[(4 * b + 1) * kSplitElems] = wb.y;
    words[(4 * b + 2) * kSplitElems] = wb.z;
    words[(4 * b + 3) * kSplitElems] = wb.w;
  }
  __syncwarp();
  uint32_t t = 0;
  if (part == 0) {
    for (uint32_t sl = 0; sl < L; ++sl) perm[sl * kSplitElems] = sl;
    t = words[0] & 1u;
    for (uint32_t widx = 1; widx < L; ++widx) {   // Fisher-Yates step j = lx + 1 - widx
      const uint32_t j = L - widx;
      const uint32_t partner = __umulhi(words[widx * kSplitElems], j + 1);
      const uint32_t a = perm[j * kSplitElems];
      const uint32_t c = perm[partner * kSplitElems];
      perm[j * kSplitElems] = c;
      perm[partner * kSplitElems] = a;
    }
  }
  __syncwarp();
  t = __shfl_sync(0xffffffffu, t, base);

  // steps 1-2, then steps 3-9 over this lane's message slots
  const Lane s0 = sh0[i], s1 = sh1[i];
  const Lane f0 = (t ? ring_neg(s0, mask) : s0) >> k.c;   // shifted by c for step 3
  const Lane nf1 = (t ? s1 : ring_neg(s1, mask)) >> k.c;
  uint32_t any_zero = 0;
  const StreamPhilox mask_stream(ep, kPair01, kPurMask, rk);
  for (uint32_t slot = part; slot < L; slot += kSplit) {
    uint32_t w0, w1;
    const U32x4 rz = mask_stream.block((uint64_t)kPhiloxM1 * slot, rk);
    any_zero |= slot_zero_test<LX, SHORT>(k, f0, nf1, perm[slot * kSplitElems], rz, w0, w1);
  }
  any_zero |= __shfl_xor_sync(0xffffffffu, any_zero, 1);
  any_zero |= __shfl_xor_sync(0xffffffffu, any_zero, 2);
  const uint32_t dprime = any_zero;

  Lane out0, out1;
  if (!RELU) {
    // steps 10-11 (lane 0 finishes)
    const U32x4 rb = ep.block_at(kPair02, kPurReply, 0, rk);
    const Lane d0 = block_elem<Lane>(rb, 0) & mask;
    const Lane d1 = ((Lane)dprime - d0) & mask;
    out0 = t ? (Lane)((Lane)1 - d0) & mask : d0;
    out1 = t ? ring_neg(d1, mask) : d1;
  } else {
    // Alg. relu: the triple's blocks are drawn by lanes 0, 1 (and 2 for l > 32)
    const U32x4 mine = part == 0 ? ep.block_at(kPair02, kPurReluTriple, 0, rk)
                       : part == 1 ? ep.block_at(kPair12, kPurReluTriple, 0, rk)
                                   : ep.block_at(kPair02, kPurReluTriple, 1, rk);
    U32x4 q1, q2;
    q1.x = __shfl_sync(0xffffffffu, mine.x, base + 1);
    q1.y = __shfl_sync(0xffffffffu, mine.y, base + 1);
    q1.z = __shfl_sync(0xffffffffu, mine.z, base + 1);
    q1.w = __shfl_sync(0xffffffffu, mine.w, base + 1);
    q2.x = __shfl_sync(0xffffffffu, mine.x, base + 2);
    q2.y = __shfl_sync(0xffffffffu, mine.y, base + 2);
    q2.z = q2.w = 0u;
    const Triple<Lane> T = triple_from_blocks<Lane>(mine, q1, q2, mask);
    const Lane c1 = (Lane)((T.a0 + T.a1) * (T.b0 + T.b1) - T.c0) & mask;
    const Lane e = (Lane)((Lane)dprime - T.b0 - T.b1) & mask;
    const Lane d = (Lane)((s0 - T.a0) + (s1 - T.a1)) & mask;
    const Lane xd0 = (Lane)(d * (e + T.b0) + e * T.a0 + T.c0) & mask;
    const Lane xd1 = (Lane)(d * T.b1 + e * T.a1 + c1) & mask;
    out0 = t ? (Lane)(s0 - xd0) & mask : xd0;
    out1 = t ? (Lane)(s1 - xd1) & mask : xd1;
  }
  if (part == 0 && valid) {
    o0[i] = out0;
    o1[i] = out1;
  }
}

template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT>
cudaError_t launch_t(const ReluConsts& k, const void* sh0, const void* sh1, uint64_t n, void* o0,
                     void* o1, const AuditPtrs& aud, int num_sms, cudaStream_t s) {
  const uint64_t grid = (n + kBlock - 1) / kBlock;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  if (!AUDIT) {
    // the split kernel's time grows with n from a few microseconds; the
    // element-per-thread kernel's is one element's latency up to a full
    // wave: about 7.5 us below one CTA per SM at lx = 24, rising to 12 and
    // 17.5 us as CTAs share the SMs.  On GB300 they cross near 0.3 waves of
    // the split kernel (about 1.2e4 elements at lx = 24).
    static const int split_per_sm = [] {   // a property of the kernel on this architecture
      int v = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, relu_split_kernel<Lane, LX, SHORT, RELU>,
                                                    kBlock, 0);
      return v < 1 ? 1 : v;
    }();
    const uint64_t split_grid = (n + kSplitElems - 1) / kSplitElems;
    if (10 * split_grid <= 3ull * (uint64_t)num_sms * (uint64_t)split_per_sm) {   // 0.3 waves
      relu_split_kernel<Lane, LX, SHORT, RELU><<<(unsigned)split_grid, kBlock, 0, s>>>(
          k, static_cast<const Lane*>(sh0), static_cast<const Lane*>(sh1), n,
          static_cast<Lane*>(o0), static_cast<Lane*>(o1));
      return cudaGetLastError();
    }
  }
  relu_kernel<Lane, LX, SHORT, RELU, AUDIT><<<(unsigned)grid, kBlock, 0, s>>>(
      k, static_cast<const Lane*>(sh0), static_cast<const Lane*>(sh1), n, static_cast<Lane*>(o0),
      static_cast<Lane*>(o1), aud);
  return cudaGetLastError();
}

template <typename Lane, bool RELU, bool AUDIT>
cudaError_t launch_lx(const ReluConsts& k, const void* sh0, const void* sh1, uint64_t n,
                      void* o0, void* o1, const AuditPtrs& aud, int num_sms, cudaStream_t s) {
  const bool shrt = sizeof(Lane) == 8 && k.c + k.lx < 32;
  switch (k.lx) {
    case 24:
      return shrt ? launch_t<Lane, 24, true, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
                  : launch_t<Lane, 24, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
    case 14: return launch_t<Lane, 14, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
    case 9: return launch_t<Lane, 9, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
    case 7:
      return shrt ? launch_t<Lane, 7, true, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
                  : launch_t<Lane, 7, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
    default: return launch_t<Lane, 0, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
  }
}

// ---------------------------------------------------------------------------
// Fused step: Beaver product -> both truncations -> ReLU, one element per
// thread.  The product and the truncated shares never leave registers unless
// the caller asks for them, so the step moves 32 bytes in and 32 bytes out per
// element (l = 64) instead of the 176 of four separate kernels.  The input and
// output pointers may also be mapped pinned host memory: the loads and stores
// then cross the host link inside the kernel while the multiplier-bound body
// of other warps hides their latency.
// ---------------------------------------------------------------------------
template <typename Lane, int LX, bool SHORT>
__global__ void __launch_bounds__(kBlock, (relu_min_ctas<Lane, LX, SHORT, false>()))
    linear_relu_kernel(const LinearConsts c, const LinearIo io, uint64_t n) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  __shared__ uint64_t r2_s[kMaxSlots + 2];   // the ReLU's table, then the product's (b = 0, 1)
  uint32_t* perm = perm_s + threadIdx.x;
  if (threadIdx.x < kMaxSlots)
    r2_s[threadIdx.x] = round2_product(c.k.tensor_id, threadIdx.x, c.k.rk);
  else if (threadIdx.x < kMaxSlots + 2)
    r2_s[threadIdx.x] = round2_product(c.mul_tid, threadIdx.x - kMaxSlots, c.k.rk);
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const uint64_t elem = c.k.elem_base + i;
  const Lane mask = (Lane)c.k.ring_mask;
  Lane p0, p1;
  beaver_mul<Lane>(ElemPhilox(elem, c.mul_tid), c.k.rk, mask,
                   static_cast<const Lane*>(io.x0)[i], static_cast<const Lane*>(io.x1)[i],
                   static_cast<const Lane*>(io.y0)[i], static_cast<const Lane*>(io.y1)[i], p0, p1,
                   r2_s + kMaxSlots);
  // Alg. smltrc: P0 cut([z]_0, k); P1 2^l - cut(2^l - [z]_1, k)
  const Lane hi0 = p0 >> c.trunc;
  const Lane hi1 = ring_neg<Lane>(p1, mask) >> c.trunc;
  const Lane t0 = hi0;
  const Lane t1 = ring_neg<Lane>(hi1, mask);
  if (io.prod0) {
    static_cast<Lane*>(io.prod0)[i] = p0;
    static_cast<Lane*>(io.prod1)[i] = p1;
  }
  if (io.trc0) {
    static_cast<Lane*>(io.trc0)[i] = t0;
    static_cast<Lane*>(io.trc1)[i] = t1;
  }
  // Alg. newtrc2 with k1 = k, k2 = 0: the same cuts, reduced mod 2^(l-k)
  if (io.det0) {
    const uint64_t dm = c.det_mask;
    const uint64_t d0 = (uint64_t)hi0 & dm, d1 = (0ull - (uint64_t)hi1) & dm;
    if (c.det_wide) {
      static_cast<uint64_t*>(io.det0)[i] = d0;
      static_cast<uint64_t*>(io.det1)[i] = d1;
    } else {
      static_cast<uint32_t*>(io.det0)[i] = (uint32_t)d0;
      static_cast<uint32_t*>(io.det1)[i] = (uint32_t)d1;
    }
  }
  Lane r0, r1;
  bicoptor_element<Lane, LX, SHORT, true, false>(c.k, c.k.rk, c.k.tensor_id, t0, t1, elem, perm,
                                                 r0, r1, AuditPtrs{}, i, r2_s);
  static_cast<Lane*>(io.relu0)[i] = r0;
  static_cast<Lane*>(io.relu1)[i] = r1;
}

template <typename Lane, int LX, bool SHORT>
cudaError_t launch_linear_t(const LinearConsts& c, const LinearIo& io, uint64_t n,
                            cudaStream_t s) {
  const uint64_t grid = (n + kBlock - 1) / kBlock;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  linear_relu_kernel<Lane, LX, SHORT><<<(unsigned)grid, kBlock, 0, s>>>(c, io, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Alg. drelu2 (RSS DReLU) and the RSS ReLU: replicated components x0, x1, x2
// (P0 holds 0 and 1, P1 holds 1 and 2, P2 holds 2 and 0).  Per element:
// preprocessing [t] (zero sharing from seed012 plus t), [s] (s from seed2),
// [s xor t] via the replicated product; Alg. drelu steps 1-9 between P0
// ([x]_0 + [x]_1) and P1 ([x]_2); P2's d'' = s xor DReLU'; the local finish
// and, for ReLU, the replicated product [x][DReLU].
// ---------------------------------------------------------------------------

template <typename Lane>
__device__ __forceinline__ void draw3(const ElemPhilox& ep, uint32_t pair, uint32_t purpose,
                                      Lane mask, const RoundKeys& rk, const uint64_t* r2,
                                      Lane out[3]) {
  const U32x4 q0 = ep.block_tab(pair, purpose, 0, r2, rk);
  if (sizeof(Lane) == 4) {
    out[0] = (Lane)q0.x & mask;
    out[1] = (Lane)q0.y & mask;
    out[2] = (Lane)q0.z & mask;
  } else {
    const U32x4 q1 = ep.block_tab(pair, purpose, 1, r2, rk);
    out[0] = block_elem<Lane>(q0, 0) & mask;
    out[1] = block_elem<Lane>(q0, 1) & mask;
    out[2] = block_elem<Lane>(q1, 0) & mask;
  }
}

template <typename Lane>
__device__ __forceinline__ void rss_mul3(const Lane a[3], const Lane b[3], const Lane g[3],
                                         Lane mask, Lane out[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = i == 2 ? 0 : i + 1;
    out[i] = (Lane)(a[i] * b[i] + a[i] * b[j] + a[j] * b[i] + g[i] - g[j]) & mask;
  }
}

template <typename Lane, int LX, bool SHORT, bool RELU>
__global__ void __launch_bounds__(kBlock)
    rss_kernel(const ReluConsts k, const Lane* __restrict__ x0, const Lane* __restrict__ x1,
               const Lane* __restrict__ x2, uint64_t n, Lane* __restrict__ y0,
               Lane* __restrict__ y1, Lane* __restrict__ y2) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  __shared__ uint64_t r2_s[kMaxSlots];
  uint32_t* perm = perm_s + threadIdx.x;
  if (threadIdx.x < kMaxSlots) r2_s[threadIdx.x] = round2_product(k.tensor_id, threadIdx.x, k.rk);
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const Lane mask = (Lane)k.ring_mask;
  const uint64_t elem = k.elem_base + i;
  const Lane X[3] = {x0[i], x1[i], x2[i]};
  Lane dp, t;
  const AuditPtrs none{};
  bicoptor_element<Lane, LX, SHORT, false, false, true>(k, k.rk, k.tensor_id,
                                                        (Lane)(X[0] + X[1]) & mask, X[2], elem,
                                                        perm, dp, t, none, i, r2_s);
  const ElemPhilox ep(elem, k.tensor_id);
  Lane al[3], S[3], T[3], g[3], ST[3], Xs[3], Y[3];
  draw3<Lane>(ep, kPair012, kPurRssT, mask, k.rk, r2_s, al);
  T[0] = (Lane)(al[0] - al[2]) & mask;
  T[1] = (Lane)(al[1] - al[0] + t) & mask;
  T[2] = (Lane)(al[2] - al[1]) & mask;
  const Lane sbit = (Lane)(ep.block_tab(kPair2, kPurRssS, 0, r2_s, k.rk).x & 1u);
  S[1] = block_elem<Lane>(ep.block_tab(kPair012, kPurRssS, 0, r2_s, k.rk), 0) & mask;
  S[2] = block_elem<Lane>(ep.block_tab(kPair12, kPurRssS, 0, r2_s, k.rk), 0) & mask;
  S[0] = (Lane)(sbit - S[1] - S[2]) & mask;                          // P2 -> P0
  draw3<Lane>(ep, kPair012, kPurRssZ, mask, k.rk, r2_s, g);
  rss_mul3<Lane>(S, T, g, mask, ST);
#pragma unroll
  for (int j = 0; j < 3; ++j) Xs[j] = (Lane)(S[j] + T[j] - 2 * ST[j]) & mask;   // [s xor t]
  const Lane dd = sbit ^ dp;                                         // d'' (P2 -> P0, P1)
#pragma unroll
  for (int j = 0; j < 3; ++j) Y[j] = (Lane)(Xs[j] - 2 * dd * Xs[j] + (j == 0 ? dd : 0)) & mask;
  if (RELU) {
    Lane gr[3], Z[3];
    draw3<Lane>(ep, kPair012, kPurRssZr, mask, k.rk, r2_s, gr);
    rss_mul3<Lane>(X, Y, gr, mask, Z);
    y0[i] = Z[0];
    y1[i] = Z[1];
    y2[i] = Z[2];
  } else {
    y0[i] = Y[0];
    y1[i] = Y[1];
    y2[i] = Y[2];
  }
}

template <typename Lane, int LX, bool SHORT, bool RELU>
cudaError_t launch_rss_t(const ReluConsts& k, const void* const* x, uint64_t n, void* const* y,
                         cudaStream_t s) {
  const uint64_t grid = (n + kBlock - 1) / kBlock;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  rss_kernel<Lane, LX, SHORT, RELU><<<(unsigned)grid, kBlock, 0, s>>>(
      k, static_cast<const Lane*>(x[0]), static_cast<const Lane*>(x[1]),
      static_cast<const Lane*>(x[2]), n, static_cast<Lane*>(y[0]), static_cast<Lane*>(y[1]),
      static_cast<Lane*>(y[2]));
  return cudaGetLastError();
}

template <typename Lane, bool RELU>
cudaError_t launch_rss_lx(const ReluConsts& k, const void* const* x, uint64_t n, void* const* y,
                          cudaStream_t s) {
  if (k.lx == 24 && sizeof(Lane) == 8 && k.c + k.lx < 32)
    return launch_rss_t<Lane, 24, true, RELU>(k, x, n, y, s);
  return launch_rss_t<Lane, 0, false, RELU>(k, x, n, y, s);
}

}  // namespace

cudaError_t launch_rss(const ReluConsts& k, bool relu, const void* const* x, uint64_t n,
                       void* const* y, cudaStream_t s) {
  if (k.ring_bits > 32)
    return relu ? launch_rss_lx<uint64_t, true>(k, x, n, y, s)
                : launch_rss_lx<uint64_t, false>(k, x, n, y, s);
  return relu ? launch_rss_lx<uint32_t, true>(k, x, n, y, s)
              : launch_rss_lx<uint32_t, false>(k, x, n, y, s);
}

cudaError_t launch_relu(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                        uint64_t n, void* o0, void* o1, const AuditPtrs& aud, int num_sms,
                        cudaStream_t s) {
  const bool lane64 = k.ring_bits > 32;
  const bool audit = aud.any();
  if (lane64) {
    if (relu) {
      return audit ? launch_lx<uint64_t, true, true>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
                   : launch_lx<uint64_t, true, false>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
    }
    return audit ? launch_lx<uint64_t, false, true>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
                 : launch_lx<uint64_t, false, false>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
  }
  if (relu) {
    return audit ? launch_lx<uint32_t, true, true>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
                 : launch_lx<uint32_t, true, false>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
  }
  return audit ? launch_lx<uint32_t, false, true>(k, sh0, sh1, n, o0, o1, aud, num_sms, s)
               : launch_lx<uint32_t, false, false>(k, sh0, sh1, n, o0, o1, aud, num_sms, s);
}

cudaError_t launch_linear_relu(const LinearConsts& c, const LinearIo& io, uint64_t n,
                               cudaStream_t s) {
  const ReluConsts& k = c.k;
  if (k.ring_bits > 32) {
    const bool shrt = k.c + k.lx < 32;
    switch (k.lx) {
      case 24:
        return shrt ? launch_linear_t<uint64_t, 24, true>(c, io, n, s)
                    : launch_linear_t<uint64_t, 24, false>(c, io, n, s);
      default: return launch_linear_t<uint64_t, 0, false>(c, io, n, s);
    }
  }
  switch (k.lx) {
    case 14: return launch_linear_t<uint32_t, 14, false>(c, io, n, s);
    case 9: return launch_linear_t<uint32_t, 9, false>(c, io, n, s);
    default: return launch_linear_t<uint32_t, 0, false>(c, io, n, s);
  }
}

}  // namespace bc
