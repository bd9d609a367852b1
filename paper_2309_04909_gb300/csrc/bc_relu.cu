// Fused Bicoptor 2.0 DReLU / ReLU kernels (Alg. drelu, Alg. relu).
//
// One thread owns one element at a time and runs, in registers, the local
// work of all three parties:
//   P0, P1  steps 1-2   flip both shares by (-1)^t, t from seed01
//           step 3      windowed deterministic truncation (Alg. newtrc2) at
//                       every key-bit position i = 0..lx
//           step 4      pair sums v_i = u_i + u_(i+1) - 1
//           step 5      Alg. modswitch into Z_p
//           step 6      seed01 shuffle (Fisher-Yates, staged in shared memory)
//           step 7-8    mask by r_k in Z_p^*, reshare by z_k
//   P2      step 9      reconstruct each w_k and test it for zero
//           step 10     reply: [DReLU']_1 to P1 (DReLU) or e = DReLU' - b (ReLU)
//   P0, P1  step 11     unflip (DReLU) / Beaver finish (ReLU)
// The lx+1 windows are never stored: message slot k recomputes the window of
// the index i = perm[k] from the two shares, so the l-fold expansion of the
// paper's step 3 costs two funnel shifts per slot and no memory traffic.
// Draws shared by P0 and P1 (everything from seed01) are generated once per
// element and used by both simulated parties.
#include "bc_internal.h"

// Tuning knobs of the fused kernel (compile-time): unroll of the message-slot
// loop and the minimum resident CTAs per SM requested from the register
// allocator (0 = let it choose).
#ifndef BC_SLOT_UNROLL
#define BC_SLOT_UNROLL 2
#endif
#ifndef BC_RELU_MIN_CTAS
#define BC_RELU_MIN_CTAS 0
#endif

namespace bc {
namespace {

constexpr int kSlotUnroll = BC_SLOT_UNROLL;

template <int LX, bool WIDE>
struct SlotMath;

// p fits in 31 bits (lx <= 30): sums of two residues stay below 2^32.
template <int LX>
struct SlotMath<LX, false> {
  static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t s = a + b;
    const uint32_t d = s - p;
    return d < s ? d : s;   // s >= p  <=>  s - p does not wrap
  }
  static __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t d = a - b;
    return a >= b ? d : d + p;
  }
};
template <int LX>
struct SlotMath<LX, true> {
  static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b, uint32_t p) {
    return add_mod(a, b, p);
  }
  static __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b, uint32_t p) {
    return sub_mod(a, b, p);
  }
};

template <typename Lane>
__device__ __forceinline__ void store_lane(void* base, uint64_t i, Lane v) {
  reinterpret_cast<Lane*>(base)[i] = v;
}

// The Beaver triple of the ReLU product for one element (Alg. relu
// preprocessing): a0,b0,c0 from seed02, a1,b1 from seed12.
template <typename Lane>
struct Triple {
  Lane a0, b0, c0, a1, b1;
};

template <typename Lane>
__device__ __forceinline__ Triple<Lane> draw_triple(const ElemPhilox& ep, uint32_t purpose,
                                                    Lane mask, const RoundKeys& rk) {
  Triple<Lane> T;
  const U32x4 q0 = ep.block_at(kPair02, purpose, 0, rk);
  const U32x4 q1 = ep.block_at(kPair12, purpose, 0, rk);
  if (sizeof(Lane) == 4) {
    T.a0 = (Lane)q0.x;
    T.b0 = (Lane)q0.y;
    T.c0 = (Lane)q0.z;
  } else {
    const U32x4 q2 = ep.block_at(kPair02, purpose, 1, rk);
    T.a0 = block_elem<Lane>(q0, 0);
    T.b0 = block_elem<Lane>(q0, 1);
    T.c0 = block_elem<Lane>(q2, 0);
  }
  T.a1 = block_elem<Lane>(q1, 0);
  T.b1 = block_elem<Lane>(q1, 1);
  T.a0 &= mask; T.b0 &= mask; T.c0 &= mask; T.a1 &= mask; T.b1 &= mask;
  return T;
}

// The 32 window bits starting at bit sh of a lane.  SHORT: sh < 32 is known
// (c + lx < 32), so a single funnel shift of the two halves suffices.
template <bool SHORT>
__device__ __forceinline__ uint32_t window32(uint64_t a, uint32_t sh) {
  if (SHORT) return __funnelshift_r((uint32_t)a, (uint32_t)(a >> 32), sh);
  return (uint32_t)(a >> sh);
}
template <bool SHORT>
__device__ __forceinline__ uint32_t window32(uint32_t a, uint32_t sh) {
  return a >> sh;
}

// Alg. drelu / Alg. relu for one element.  `perm` points at this thread's
// column of the shared-memory shuffle table (stride kBlock words).
// DPONLY: stop after P2's step 9 and return DReLU' in out0 and t in out1
// (the RSS protocol finishes differently).
template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT, bool DPONLY = false>
__device__ __forceinline__ void bicoptor_element(const ReluConsts& k, const RoundKeys& rk,
                                                 uint32_t tensor_id, Lane s0, Lane s1,
                                                 uint64_t elem, uint32_t* perm, Lane& out0,
                                                 Lane& out1, const AuditPtrs& aud,
                                                 uint64_t out_idx) {
  constexpr bool kWide = (LX == 0) || (LX > 30);
  using M = SlotMath<LX, kWide>;
  const uint32_t lx = LX ? (uint32_t)LX : k.lx;
  const uint32_t L = lx + 1;
  const Lane mask = (Lane)k.ring_mask;
  const uint32_t p = k.mp.p;
  const ElemPhilox ep(elem, tensor_id);

  // ---- seed01 stream: t (step 1) and the shuffle words (step 6) ----------
#pragma unroll
  for (uint32_t s = 0; s < (LX ? (uint32_t)(LX + 1) : (uint32_t)kMaxSlots); ++s) {
    if (LX || s < L) perm[s * kBlock] = s;
  }
  uint32_t t = 0;
  const uint32_t nblk = (L + 3) >> 2;
  const StreamPhilox perm_stream(ep, kPair01, kPurPerm, rk);
#pragma unroll
  for (uint32_t b = 0; b < (LX ? (uint32_t)((LX + 4) >> 2) : 8u); ++b) {
    if (!LX && b >= nblk) break;
    const U32x4 wb = perm_stream.block((uint64_t)kPhiloxM1 * b, rk);
    const uint32_t ws[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t widx = 4 * b + q;
      if (widx == 0) {
        t = ws[0] & 1u;
      } else if (widx < L) {
        // Fisher-Yates step j = lx + 1 - widx: partner = floor(W (j+1) / 2^32)
        const uint32_t j = L - widx;
        const uint32_t partner = __umulhi(ws[q], j + 1);
        const uint32_t a = perm[j * kBlock];
        const uint32_t c = perm[partner * kBlock];
        perm[j * kBlock] = c;
        perm[partner * kBlock] = a;
      }
    }
  }

  // ---- steps 1-2: flip by (-1)^t --------------------------------------------
  const Lane f0 = t ? ring_neg(s0, mask) : s0;
  const Lane nf1 = t ? s1 : ring_neg(s1, mask);   // 2^l - [x]_1 of the flipped share

  // ---- steps 3-9 over message slots k ----------------------------------------
  uint32_t any_zero = 0;
  const StreamPhilox mask_stream(ep, kPair01, kPurMask, rk);
  uint64_t mb = 0;   // M1 * slot, the round-1 product of the slot's mask block
#pragma unroll kSlotUnroll
  for (uint32_t slot = 0; slot < L; ++slot, mb += kPhiloxM1) {
    const uint32_t i = perm[slot * kBlock];
    const uint32_t sh = k.c + i;
    const uint32_t y0 = window32<SHORT>(f0, sh);
    const uint32_t y1 = window32<SHORT>(nf1, sh);
    const uint32_t next_mask = (i < lx) ? k.mx : 0u;   // u_(lx+1) := 0
    // steps 3-4: P0 v = u_i + u_(i+1) - 1, P1 v = u_i + u_(i+1) with u = -cut(-x1)
    const uint32_t v0 = ((y0 & k.mx) + ((y0 >> 1) & next_mask) - 1u) & k.mx;
    const uint32_t v1 = (0u - (y1 & k.mx) - ((y1 >> 1) & next_mask)) & k.mx;
    // step 5: Alg. modswitch
    const uint32_t m0 = v0 ? v0 : k.two_lx;
    const uint32_t m1 = v1 + k.p_minus_2lx;
    // step 7: rho_k, z_k from the slot's seed01 block; the mask r_k =
    // rho_k 2^-32 mod p, so one Montgomery product m rho 2^-32 is m r_k
    const U32x4 rz = mask_stream.block(mb, rk);
    const uint32_t rho = 1u + mulhi_64x32(rz.x, rz.y, k.mp.pm1);
    const uint32_t z = mulhi_64x32(rz.z, rz.w, p);
    uint32_t w0 = mont_mul<kWide>(m0, rho, k.mp);
    uint32_t w1 = mont_mul<kWide>(m1, rho, k.mp);
    // step 8: reshare (P0 adds z_k, P1 subtracts it) and send to P2
    w0 = M::add(w0, z, p);
    w1 = M::sub(w1, z, p);
    if (AUDIT) {
      if (aud.w0) aud.w0[out_idx * L + slot] = w0;
      if (aud.w1) aud.w1[out_idx * L + slot] = w1;
    }
    // step 9: P2 reconstructs w_k and tests it
    any_zero |= (M::add(w0, w1, p) == 0u) ? 1u : 0u;
  }
  const uint32_t dprime = any_zero;
  if (DPONLY) {
    out0 = (Lane)dprime;
    out1 = (Lane)t;
    return;
  }

  if (!RELU) {
    // step 10: [DReLU']_0 = d0 from seed02 (P0 derives it), [DReLU']_1 to P1
    const U32x4 rb = ep.block_at(kPair02, kPurReply, 0, rk);
    const Lane d0 = block_elem<Lane>(rb, 0) & mask;
    const Lane d1 = ((Lane)dprime - d0) & mask;
    // step 11: [DReLU] = [DReLU' xor t], the public t added by P0
    out0 = t ? (Lane)((Lane)1 - d0) & mask : d0;
    out1 = t ? ring_neg(d1, mask) : d1;
    if (AUDIT && aud.reply) store_lane<Lane>(aud.reply, out_idx, d1);
  } else {
    const Triple<Lane> T = draw_triple<Lane>(ep, kPurReluTriple, mask, rk);
    const Lane c1 = (Lane)((T.a0 + T.a1) * (T.b0 + T.b1) - T.c0) & mask;   // P2 -> P1 (pre)
    const Lane e = (Lane)((Lane)dprime - T.b0 - T.b1) & mask;             // P2 -> P0, P1
    const Lane open0 = (Lane)(s0 - T.a0) & mask;                          // P0 -> P1
    const Lane open1 = (Lane)(s1 - T.a1) & mask;                          // P1 -> P0
    const Lane d = (Lane)(open0 + open1) & mask;
    const Lane xd0 = (Lane)(d * (e + T.b0) + e * T.a0 + T.c0) & mask;
    const Lane xd1 = (Lane)(d * T.b1 + e * T.a1 + c1) & mask;
    out0 = t ? (Lane)(s0 - xd0) & mask : xd0;
    out1 = t ? (Lane)(s1 - xd1) & mask : xd1;
    if (AUDIT) {
      if (aud.reply) store_lane<Lane>(aud.reply, out_idx, e);
      if (aud.open0) store_lane<Lane>(aud.open0, out_idx, open0);
      if (aud.open1) store_lane<Lane>(aud.open1, out_idx, open1);
      if (aud.pre_c1) store_lane<Lane>(aud.pre_c1, out_idx, c1);
    }
  }
  if (AUDIT) {
    if (aud.t) aud.t[out_idx] = (uint8_t)t;
    if (aud.dprime) aud.dprime[out_idx] = (uint8_t)dprime;
  }
}

// One element per thread; the grid covers the tensor once, so the CTA
// scheduler hands out work as CTAs retire (no static tail).
template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT>
__global__ void __launch_bounds__(kBlock, BC_RELU_MIN_CTAS)
    relu_kernel(const ReluConsts k, const Lane* __restrict__ sh0, const Lane* __restrict__ sh1,
                uint64_t n, Lane* __restrict__ o0, Lane* __restrict__ o1, const AuditPtrs aud) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  uint32_t* perm = perm_s + threadIdx.x;
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  Lane r0, r1;
  bicoptor_element<Lane, LX, SHORT, RELU, AUDIT>(k, k.rk, k.tensor_id, sh0[i], sh1[i],
                                                 k.elem_base + i, perm, r0, r1, aud, i);
  o0[i] = r0;
  o1[i] = r1;
}

template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT>
cudaError_t launch_t(const ReluConsts& k, const void* sh0, const void* sh1, uint64_t n, void* o0,
                     void* o1, const AuditPtrs& aud, cudaStream_t s) {
  const uint64_t grid = (n + kBlock - 1) / kBlock;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  relu_kernel<Lane, LX, SHORT, RELU, AUDIT><<<(unsigned)grid, kBlock, 0, s>>>(
      k, static_cast<const Lane*>(sh0), static_cast<const Lane*>(sh1), n, static_cast<Lane*>(o0),
      static_cast<Lane*>(o1), aud);
  return cudaGetLastError();
}

template <typename Lane, bool RELU, bool AUDIT>
cudaError_t launch_lx(const ReluConsts& k, const void* sh0, const void* sh1, uint64_t n,
                      void* o0, void* o1, const AuditPtrs& aud, cudaStream_t s) {
  const bool shrt = sizeof(Lane) == 8 && k.c + k.lx < 32;
  switch (k.lx) {
    case 24:
      return shrt ? launch_t<Lane, 24, true, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s)
                  : launch_t<Lane, 24, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s);
    case 14: return launch_t<Lane, 14, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s);
    case 9: return launch_t<Lane, 9, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s);
    case 7:
      return shrt ? launch_t<Lane, 7, true, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s)
                  : launch_t<Lane, 7, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s);
    default: return launch_t<Lane, 0, false, RELU, AUDIT>(k, sh0, sh1, n, o0, o1, aud, s);
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
__global__ void __launch_bounds__(kBlock, BC_RELU_MIN_CTAS)
    linear_relu_kernel(const LinearConsts c, const LinearIo io, uint64_t n) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  uint32_t* perm = perm_s + threadIdx.x;
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const uint64_t elem = c.k.elem_base + i;
  const Lane mask = (Lane)c.k.ring_mask;
  Lane p0, p1;
  beaver_mul<Lane>(ElemPhilox(elem, c.mul_tid), c.k.rk, mask,
                   static_cast<const Lane*>(io.x0)[i], static_cast<const Lane*>(io.x1)[i],
                   static_cast<const Lane*>(io.y0)[i], static_cast<const Lane*>(io.y1)[i], p0, p1);
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
                                                 r0, r1, AuditPtrs{}, i);
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
// Batched form: one persistent launch per (lane width, key bits) class over
// that class's range of a tile table of many tensors.  Every warp takes the
// next tile from the class's atomic counter on its own (no block barrier, no
// waits), so uneven tensors balance across the SMs down to one tile per warp;
// per-class kernels keep the register allocation of a single variant.
// ---------------------------------------------------------------------------

template <typename Lane, int LX, bool SHORT, bool RELU>
__device__ __forceinline__ void run_tile(const ReluConsts& k, const BatchTensor& bt,
                                         uint64_t start, uint32_t count, uint32_t lane,
                                         uint32_t* perm) {
  const Lane* sh0 = static_cast<const Lane*>(bt.sh0);
  const Lane* sh1 = static_cast<const Lane*>(bt.sh1);
  Lane* o0 = static_cast<Lane*>(bt.o0);
  Lane* o1 = static_cast<Lane*>(bt.o1);
  const AuditPtrs none{};
#pragma unroll 1
  for (uint32_t j = lane; j < count; j += 32) {
    const uint64_t i = start + j;
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, RELU, false>(k, k.rk, bt.tensor_id, sh0[i], sh1[i],
                                                   bt.elem_offset + i, perm, r0, r1, none, i);
    o0[i] = r0;
    o1[i] = r1;
  }
}

template <typename Lane, int LX, bool SHORT>
__global__ void __launch_bounds__(kBlock)
    relu_batch_kernel(const ReluConsts k, const BatchTensor* __restrict__ tensors,
                      const BatchTile* __restrict__ tiles, uint32_t begin, uint32_t end,
                      unsigned int* __restrict__ counter, int* __restrict__ status) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  uint32_t* perm = perm_s + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    uint32_t tile = 0;
    if (lane == 0) tile = begin + atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= end) break;
    const BatchTile tl = tiles[tile];
    const BatchTensor bt = tensors[tl.tensor];
    if (tl.start + tl.count > bt.n) {   // a malformed table: record, skip
      if (lane == 0) atomicExch(status, BC_ECHECK);
      continue;
    }
    if (bt.op == BC_OP_DRELU) run_tile<Lane, LX, SHORT, false>(k, bt, tl.start, tl.count, lane, perm);
    else run_tile<Lane, LX, SHORT, true>(k, bt, tl.start, tl.count, lane, perm);
  }
}

// Grid schedule: one CTA per tile of at most kBlock elements, one element per
// thread, no loop; the hardware CTA scheduler hands out the tiles.
template <typename Lane, int LX, bool SHORT>
__global__ void __launch_bounds__(kBlock)
    relu_batch_grid_kernel(const ReluConsts k, const BatchTensor* __restrict__ tensors,
                           const BatchTile* __restrict__ tiles, uint32_t begin,
                           int* __restrict__ status) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  uint32_t* perm = perm_s + threadIdx.x;
  const BatchTile tl = tiles[begin + blockIdx.x];
  const BatchTensor bt = tensors[tl.tensor];
  if (tl.count > kBlock || tl.start + tl.count > bt.n) {   // a malformed table: record, skip
    if (threadIdx.x == 0) atomicExch(status, BC_ECHECK);
    return;
  }
  if (threadIdx.x >= tl.count) return;
  const uint64_t i = tl.start + threadIdx.x;
  const AuditPtrs none{};
  if (bt.op == BC_OP_DRELU) {
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, false, false>(
        k, k.rk, bt.tensor_id, static_cast<const Lane*>(bt.sh0)[i],
        static_cast<const Lane*>(bt.sh1)[i], bt.elem_offset + i, perm, r0, r1, none, i);
    static_cast<Lane*>(bt.o0)[i] = r0;
    static_cast<Lane*>(bt.o1)[i] = r1;
  } else {
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, true, false>(
        k, k.rk, bt.tensor_id, static_cast<const Lane*>(bt.sh0)[i],
        static_cast<const Lane*>(bt.sh1)[i], bt.elem_offset + i, perm, r0, r1, none, i);
    static_cast<Lane*>(bt.o0)[i] = r0;
    static_cast<Lane*>(bt.o1)[i] = r1;
  }
}

template <typename Lane, int LX, bool SHORT>
cudaError_t launch_group(const BatchGroup& g, const BatchTensor* tensors, const BatchTile* tiles,
                         unsigned int* counter, int* status, int num_sms, int ctas_per_sm,
                         cudaStream_t s) {
  if (ctas_per_sm < 0) {   // grid schedule
    const uint32_t ntiles = g.end - g.begin;
    if (ntiles == 0) return cudaSuccess;
    relu_batch_grid_kernel<Lane, LX, SHORT><<<ntiles, kBlock, 0, s>>>(g.k, tensors, tiles, g.begin,
                                                                      status);
    return cudaGetLastError();
  }
  auto kern = relu_batch_kernel<Lane, LX, SHORT>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  const uint64_t warps_needed = g.end - g.begin;             // at most one tile per warp
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t cap = (warps_needed * 32 + kBlock - 1) / kBlock;
  if (cap < grid) grid = cap;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned)grid, kBlock, 0, s>>>(g.k, tensors, tiles, g.begin, g.end, counter, status);
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
                                      Lane mask, const RoundKeys& rk, Lane out[3]) {
  const U32x4 q0 = ep.block_at(pair, purpose, 0, rk);
  if (sizeof(Lane) == 4) {
    out[0] = (Lane)q0.x & mask;
    out[1] = (Lane)q0.y & mask;
    out[2] = (Lane)q0.z & mask;
  } else {
    const U32x4 q1 = ep.block_at(pair, purpose, 1, rk);
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
  uint32_t* perm = perm_s + threadIdx.x;
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const Lane mask = (Lane)k.ring_mask;
  const uint64_t elem = k.elem_base + i;
  const Lane X[3] = {x0[i], x1[i], x2[i]};
  Lane dp, t;
  const AuditPtrs none{};
  bicoptor_element<Lane, LX, SHORT, false, false, true>(k, k.rk, k.tensor_id,
                                                        (Lane)(X[0] + X[1]) & mask, X[2], elem,
                                                        perm, dp, t, none, i);
  const ElemPhilox ep(elem, k.tensor_id);
  Lane al[3], S[3], T[3], g[3], ST[3], Xs[3], Y[3];
  draw3<Lane>(ep, kPair012, kPurRssT, mask, k.rk, al);
  T[0] = (Lane)(al[0] - al[2]) & mask;
  T[1] = (Lane)(al[1] - al[0] + t) & mask;
  T[2] = (Lane)(al[2] - al[1]) & mask;
  const Lane sbit = (Lane)(ep.block_at(kPair2, kPurRssS, 0, k.rk).x & 1u);
  S[1] = block_elem<Lane>(ep.block_at(kPair012, kPurRssS, 0, k.rk), 0) & mask;
  S[2] = block_elem<Lane>(ep.block_at(kPair12, kPurRssS, 0, k.rk), 0) & mask;
  S[0] = (Lane)(sbit - S[1] - S[2]) & mask;                          // P2 -> P0
  draw3<Lane>(ep, kPair012, kPurRssZ, mask, k.rk, g);
  rss_mul3<Lane>(S, T, g, mask, ST);
#pragma unroll
  for (int j = 0; j < 3; ++j) Xs[j] = (Lane)(S[j] + T[j] - 2 * ST[j]) & mask;   // [s xor t]
  const Lane dd = sbit ^ dp;                                         // d'' (P2 -> P0, P1)
#pragma unroll
  for (int j = 0; j < 3; ++j) Y[j] = (Lane)(Xs[j] - 2 * dd * Xs[j] + (j == 0 ? dd : 0)) & mask;
  if (RELU) {
    Lane gr[3], Z[3];
    draw3<Lane>(ep, kPair012, kPurRssZr, mask, k.rk, gr);
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
  (void)num_sms;
  const bool lane64 = k.ring_bits > 32;
  const bool audit = aud.any();
  if (lane64) {
    if (relu) {
      return audit ? launch_lx<uint64_t, true, true>(k, sh0, sh1, n, o0, o1, aud, s)
                   : launch_lx<uint64_t, true, false>(k, sh0, sh1, n, o0, o1, aud, s);
    }
    return audit ? launch_lx<uint64_t, false, true>(k, sh0, sh1, n, o0, o1, aud, s)
                 : launch_lx<uint64_t, false, false>(k, sh0, sh1, n, o0, o1, aud, s);
  }
  if (relu) {
    return audit ? launch_lx<uint32_t, true, true>(k, sh0, sh1, n, o0, o1, aud, s)
                 : launch_lx<uint32_t, true, false>(k, sh0, sh1, n, o0, o1, aud, s);
  }
  return audit ? launch_lx<uint32_t, false, true>(k, sh0, sh1, n, o0, o1, aud, s)
               : launch_lx<uint32_t, false, false>(k, sh0, sh1, n, o0, o1, aud, s);
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

cudaError_t launch_relu_batch(const BatchTensor* tensors, const BatchTile* tiles,
                              const BatchGroup* groups, int ngroups, unsigned int* counters,
                              int* status, int num_sms, int ctas_per_sm, cudaStream_t s) {
  for (int gi = 0; gi < ngroups; ++gi) {
    const BatchGroup& g = groups[gi];
    if (g.end <= g.begin) continue;
    unsigned int* ctr = counters + gi;
    const bool lane64 = g.k.ring_bits > 32;
    cudaError_t e;
    if (lane64) {
      if (g.k.lx == 24 && g.k.c + g.k.lx < 32)
        e = launch_group<uint64_t, 24, true>(g, tensors, tiles, ctr, status, num_sms, ctas_per_sm, s);
      else
        e = launch_group<uint64_t, 0, false>(g, tensors, tiles, ctr, status, num_sms, ctas_per_sm, s);
    } else if (g.k.lx == 14) {
      e = launch_group<uint32_t, 14, false>(g, tensors, tiles, ctr, status, num_sms, ctas_per_sm, s);
    } else if (g.k.lx == 9) {
      e = launch_group<uint32_t, 9, false>(g, tensors, tiles, ctr, status, num_sms, ctas_per_sm, s);
    } else {
      e = launch_group<uint32_t, 0, false>(g, tensors, tiles, ctr, status, num_sms, ctas_per_sm, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bc
