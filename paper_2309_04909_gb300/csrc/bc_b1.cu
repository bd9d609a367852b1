// The Bicoptor 1.0-style DReLU / ReLU that Bicoptor 2.0 improves on, as the
// paper describes it by contrast (Table "compare", Sec. "sub:cmp", the notes
// on steps 3 and 4 of Alg. drelu), for an in-house comparison of
// communication and speed:
//   step 3  Alg. smltrc (SecureML) truncations in Z_{2^l} at every key-bit
//           position c + i, i = 0..lx, instead of Alg. newtrc2 in Z_{2^lx}
//   step 4  recursive sums S_i = sum_{k=i..lx} u_k, v_i = S_i - 1 (P0 holds
//           the constant), instead of adjacent pairs
//   no modulo switch: the mask r_k (a random odd element, a unit of
//   Z_{2^l}, so zero <=> zero), the reshare z_k and P2's zero test are in
//   Z_{2^l}; each party sends lx + 1 ring elements, (lx + 1) l bits
// t, the shuffle, the reply and the ReLU triple are drawn as in Bicoptor 2.0;
// the masks come from purpose tag kPurB1Mask.
//
// The recursive sums need no loop: P0's u_k is floor(a / 2^(c+k)) for its
// flipped share a, and sum_{k >= 0} floor(a / 2^k) = 2a - popcount(a), so
//   S_i = F(a >> (c+i)) - F(a >> (c+lx+1)),  F(a) = 2a - popcount(a),
// and P1's sums are the negation of the same for b = -[x]_1 of its flipped
// share.  Each message slot thus computes its sum from the two shares in a
// few instructions, like the windows of the Bicoptor 2.0 kernel.
#include "bc_element.cuh"

namespace bc {
namespace {

__device__ __forceinline__ uint64_t floor_sum(uint64_t a) {
  return 2 * a - (uint64_t)__popcll(a);
}
// a >> s for 0 <= s <= 64 (a >> 64 = 0)
__device__ __forceinline__ uint64_t shr64(uint64_t a, uint32_t s) {
  return s >= 64 ? 0 : a >> s;
}

// Steps 3-9 of one message slot whose window offset is pos (= perm[slot]):
// the recursive sums of both parties, the mask r_k and reshare z_k from the
// slot's seed01 block, and P2's zero test.  mb = M1 * slot, the round-1
// product of the slot's mask block.  a and b arrive shifted right by the key
// offset c, so the window of offset pos starts at bit pos.
template <typename Lane>
__device__ __forceinline__ uint32_t b1_slot(const ReluConsts& k, const StreamPhilox& mask_stream,
                                            const uint64_t* r2, uint32_t slot, uint64_t mb,
                                            uint32_t pos, uint64_t a, uint64_t b, uint64_t top0,
                                            uint64_t top1, uint64_t mask, Lane* w0, Lane* w1,
                                            uint64_t wi) {
  const uint64_t v0 = (floor_sum(a >> pos) - top0 - 1) & mask;      // S0 - 1 (P0)
  const uint64_t v1 = (top1 - floor_sum(b >> pos)) & mask;          // S1 = -(sum for b)
  const U32x4 rz = mask_stream.block_p0(mb, r2[slot], k.rk);
  const uint64_t r = (((uint64_t)rz.y << 32) | rz.x) | 1u;           // odd: a unit
  const uint64_t z = ((uint64_t)rz.w << 32) | rz.z;
  const uint64_t m0 = (v0 * r + z) & mask;                           // P0 -> P2
  const uint64_t m1 = (v1 * r - z) & mask;                           // P1 -> P2
  if (w0) {
    w0[wi + slot] = (Lane)m0;
    w1[wi + slot] = (Lane)m1;
  }
  return ((m0 + m1) & mask) == 0 ? 1u : 0u;                         // step 9
}

// LX: the key width as a compile-time constant (0 = read from k).  For a
// fixed width the slots run unrolled and interleaved with the shuffle (slot j
// right after the Fisher-Yates step that fixes position j), as in the
// Bicoptor 2.0 kernels, so the two protocols are compared in the same form.
template <typename Lane, bool RELU, int LX>
__global__ void __launch_bounds__(kBlock)
    b1_kernel(const ReluConsts k, const Lane* __restrict__ sh0, const Lane* __restrict__ sh1,
              uint64_t n, Lane* __restrict__ o0, Lane* __restrict__ o1, Lane* __restrict__ w0,
              Lane* __restrict__ w1) {
  __shared__ uint32_t perm_s[kMaxSlots * kBlock];
  __shared__ uint64_t r2_s[kMaxSlots];
  if (threadIdx.x < kMaxSlots) r2_s[threadIdx.x] = round2_product(k.tensor_id, threadIdx.x, k.rk);
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const RoundKeys& rk = k.rk;
  const uint32_t lx = LX ? (uint32_t)LX : k.lx, L = lx + 1;
  const uint64_t mask = k.ring_mask;
  const ElemPhilox ep(k.elem_base + i, k.tensor_id);
  uint32_t* perm = perm_s + threadIdx.x;
  const uint64_t s0 = (uint64_t)sh0[i], s1 = (uint64_t)sh1[i];
  const uint32_t top = lx + 1;   // above the windows, counted from bit c
  const StreamPhilox perm_stream(ep, kPair01, kPurPerm, rk);
  const StreamPhilox mask_stream(ep, kPair01, kPurB1Mask, rk);
  uint32_t t = 0, any_zero = 0;
  // steps 1-2: flip; P0 keeps its flipped share a, P1 b = 2^l - its flipped
  // share, both shifted right by the key offset c once for the windows
  uint64_t a = 0, b = 0, top0 = 0, top1 = 0;
  auto flip = [&](uint32_t tt) {
    a = (tt ? (0 - s0) & mask : s0) >> k.c;
    b = (tt ? s1 : (0 - s1) & mask) >> k.c;
    top0 = floor_sum(shr64(a, top));
    top1 = floor_sum(shr64(b, top));
  };

  if (LX) {
#pragma unroll
    for (uint32_t s = 0; s < L; ++s) perm[s * kBlock] = s;
#pragma unroll
    for (uint32_t blk = 0; blk < (L + 3) / 4; ++blk) {
      const U32x4 wb = perm_stream.block_p0((uint64_t)kPhiloxM1 * blk, r2_s[blk], rk);
      const uint32_t ws[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t widx = 4 * blk + q;
        if (widx == 0) {
          t = ws[0] & 1u;
          flip(t);
        } else if (widx < L) {
          const uint32_t j = L - widx;                       // step 6, then slot j
          const uint32_t partner = __umulhi(ws[q], j + 1);
          const uint32_t pa = perm[j * kBlock];
          const uint32_t pc = perm[partner * kBlock];
          perm[partner * kBlock] = pa;   // position j is final; later steps never read it
          any_zero |= b1_slot<Lane>(k, mask_stream, r2_s, j, (uint64_t)kPhiloxM1 * j, pc, a, b,
                                    top0, top1, mask, w0, w1, i * L);
        }
      }
    }
    any_zero |= b1_slot<Lane>(k, mask_stream, r2_s, 0, 0, perm[0], a, b, top0, top1, mask, w0,
                              w1, i * L);
  } else {
    // steps 1 and 6: t and the Fisher-Yates shuffle from the seed01 stream
    for (uint32_t s = 0; s < L; ++s) perm[s * kBlock] = s;
    for (uint32_t blk = 0; blk < (L + 3) >> 2; ++blk) {
      const U32x4 wb = perm_stream.block_p0((uint64_t)kPhiloxM1 * blk, r2_s[blk], rk);
      const uint32_t ws[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t widx = 4 * blk + q;
        if (widx == 0) {
          t = ws[0] & 1u;
        } else if (widx < L) {
          const uint32_t j = L - widx;
          const uint32_t partner = __umulhi(ws[q], j + 1);
          const uint32_t pa = perm[j * kBlock];
          const uint32_t pc = perm[partner * kBlock];
          perm[j * kBlock] = pc;
          perm[partner * kBlock] = pa;
        }
      }
    }
    flip(t);
    // steps 3-9 per message slot
    uint64_t mb = 0;
#pragma unroll 2
    for (uint32_t slot = 0; slot < L; ++slot, mb += kPhiloxM1)
      any_zero |= b1_slot<Lane>(k, mask_stream, r2_s, slot, mb, perm[slot * kBlock], a, b, top0,
                                top1, mask, w0, w1, i * L);
  }
  const uint32_t dprime = any_zero;
  const Lane lmask = (Lane)mask;
  Lane out0, out1;
  if (!RELU) {
    // steps 10-11 as in Bicoptor 2.0
    const Lane d0 = block_elem<Lane>(ep.block_p0(kPair02, kPurReply, 0, r2_s[0], rk), 0) & lmask;
    const Lane d1 = ((Lane)dprime - d0) & lmask;
    out0 = t ? (Lane)((Lane)1 - d0) & lmask : d0;
    out1 = t ? ring_neg(d1, lmask) : d1;
  } else {
    const Triple<Lane> T = draw_triple<Lane>(ep, kPurReluTriple, lmask, rk, r2_s);
    const Lane x0 = (Lane)s0, x1 = (Lane)s1;
    const Lane c1 = (Lane)((T.a0 + T.a1) * (T.b0 + T.b1) - T.c0) & lmask;
    const Lane e = (Lane)((Lane)dprime - T.b0 - T.b1) & lmask;
    const Lane d = (Lane)((x0 - T.a0) + (x1 - T.a1)) & lmask;
    const Lane xd0 = (Lane)(d * (e + T.b0) + e * T.a0 + T.c0) & lmask;
    const Lane xd1 = (Lane)(d * T.b1 + e * T.a1 + c1) & lmask;
    out0 = t ? (Lane)(x0 - xd0) & lmask : xd0;
    out1 = t ? (Lane)(x1 - xd1) & lmask : xd1;
  }
  o0[i] = out0;
  o1[i] = out1;
}

template <typename Lane, bool RELU>
cudaError_t launch_b1_t(const ReluConsts& k, const void* sh0, const void* sh1, uint64_t n,
                        void* o0, void* o1, void* w0, void* w1, cudaStream_t s) {
  const uint64_t grid = (n + kBlock - 1) / kBlock;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  // the key widths the comparison runs at l = 64 (lx = 24, and the paper's
  // lx = 7 with c = 24) have fixed-width kernels, as Bicoptor 2.0's do
  auto kern = b1_kernel<Lane, RELU, 0>;
  if constexpr (sizeof(Lane) == 8) {
    if (k.lx == 24) kern = b1_kernel<Lane, RELU, 24>;
    if (k.lx == 7) kern = b1_kernel<Lane, RELU, 7>;
  }
  kern<<<(unsigned)grid, kBlock, 0, s>>>(
      k, static_cast<const Lane*>(sh0), static_cast<const Lane*>(sh1), n,
      static_cast<Lane*>(o0), static_cast<Lane*>(o1), static_cast<Lane*>(w0),
      static_cast<Lane*>(w1));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_b1(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                      uint64_t n, void* o0, void* o1, void* w0, void* w1, cudaStream_t s) {
  if (k.ring_bits > 32)
    return relu ? launch_b1_t<uint64_t, true>(k, sh0, sh1, n, o0, o1, w0, w1, s)
                : launch_b1_t<uint64_t, false>(k, sh0, sh1, n, o0, o1, w0, w1, s);
  return relu ? launch_b1_t<uint32_t, true>(k, sh0, sh1, n, o0, o1, w0, w1, s)
              : launch_b1_t<uint32_t, false>(k, sh0, sh1, n, o0, o1, w0, w1, s);
}

}  // namespace bc
