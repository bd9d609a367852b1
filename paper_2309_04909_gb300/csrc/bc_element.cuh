// The per-element body of Alg. drelu / Alg. relu, shared by the single-tensor,
// fused-step and batched kernels.
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
// paper's step 3 costs two funnel shifts per slot and party (the window u_i
// and the next one, u_(i+1)) and no memory traffic.
// Draws shared by P0 and P1 (everything from seed01) are generated once per
// element and used by both simulated parties.
#pragma once
#include "bc_internal.h"

// Default unroll of the message-slot loop (compile-time).  0: the whole loop
// when the key width is a compile-time constant (every slot's block index,
// shared-memory offsets and counter become immediates, so no loop counter,
// address increment or 64-bit counter add reaches the multiplier pipe), else 2.
#ifndef BC_SLOT_UNROLL
#define BC_SLOT_UNROLL 0
#endif

// The slot loop's Z_p sums as three-input adds (1) or in their plain form (0).
// The loop is bound by the FMA-heavy pipe, which executes the integer
// multiplies; the compiler issues every two-input integer add there too (as a
// multiply-add by one), while a three-input add exists only on the integer
// ALU, which has room.  So each sum gets a third operand that is always 0 but
// comes from the kernel parameters (zero1, zero2: the compiler cannot fold
// them), a reduction x mod p of x < 2p is min(x, x - p + 0), and each
// reduction is chained on the sum it reduces so that no two-input partial
// sum is shared.  The values are unchanged.
#ifndef BC_ALU_ADDS
#define BC_ALU_ADDS 1
#endif

// For a fixed key width, interleave the shuffle with the slot loop (1: each
// slot's message right after the shuffle step that fixes its window index,
// so the shared-memory swaps overlap the multiplier work) or shuffle first
// (0).  The values are unchanged.
#ifndef BC_INTERLEAVE
#define BC_INTERLEAVE 1
#endif

namespace bc {


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

// The triple from its Philox blocks: q0 = seed02 block 0, q1 = seed12 block
// 0, q2 = seed02 block 1 (used for l > 32 only).
template <typename Lane>
__device__ __forceinline__ Triple<Lane> triple_from_blocks(const U32x4& q0, const U32x4& q1,
                                                           const U32x4& q2, Lane mask) {
  Triple<Lane> T;
  if (sizeof(Lane) == 4) {
    T.a0 = (Lane)q0.x;
    T.b0 = (Lane)q0.y;
    T.c0 = (Lane)q0.z;
  } else {
    T.a0 = block_elem<Lane>(q0, 0);
    T.b0 = block_elem<Lane>(q0, 1);
    T.c0 = block_elem<Lane>(q2, 0);
  }
  T.a1 = block_elem<Lane>(q1, 0);
  T.b1 = block_elem<Lane>(q1, 1);
  T.a0 &= mask; T.b0 &= mask; T.c0 &= mask; T.a1 &= mask; T.b1 &= mask;
  return T;
}

template <typename Lane>
__device__ __forceinline__ Triple<Lane> draw_triple(const ElemPhilox& ep, uint32_t purpose,
                                                    Lane mask, const RoundKeys& rk,
                                                    const uint64_t* r2 = nullptr) {
  const U32x4 q0 = ep.block_tab(kPair02, purpose, 0, r2, rk);
  const U32x4 q1 = ep.block_tab(kPair12, purpose, 0, r2, rk);
  const U32x4 q2 = sizeof(Lane) == 4 ? q0 : ep.block_tab(kPair02, purpose, 1, r2, rk);
  return triple_from_blocks<Lane>(q0, q1, q2, mask);
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

// Steps 3-9 of one message slot from P0's and P1's windows y0, y1 (32 bits of
// each flipped share from bit c + i, i the slot's window index): pair sums
// (Alg. newtrc2), Alg. modswitch, the mask r_k and the reshare z_k from the
// slot's seed01 block rz, and P2's reconstruction.  sh1 gives u_(i+1): 1 for
// i < lx, 33 for i = lx (a funnel shift of (0, y) clamped at 32 then gives 0,
// as u_(lx+1) := 0).  Returns P2's w_k = w0 + w1 mod p, which its zero test
// compares with 0; w0, w1 are the two messages.
template <int LX>
__device__ __forceinline__ uint32_t slot_from_windows(const ReluConsts& k, uint32_t y0,
                                                      uint32_t y1, uint32_t sh1,
                                                      const U32x4& rz, uint32_t& w0,
                                                      uint32_t& w1) {
  constexpr bool kWide = (LX == 0) || (LX > 30);
  using M = SlotMath<LX, kWide>;
  const uint32_t mx = LX ? (uint32_t)((1ull << (LX ? LX : 1)) - 1u) : k.mx;   // 2^lx - 1
  const uint32_t p = k.mp.p;
  const uint32_t n0 = __funnelshift_rc(y0, 0u, sh1), n1 = __funnelshift_rc(y1, 0u, sh1);
  // steps 3-4: P0 v = u_i + u_(i+1) - 1, P1 v = u_i + u_(i+1) with u = -cut(-x1);
  // sums mod 2^lx depend only on the low lx bits of their terms, so neither
  // u_i nor u_(i+1) needs its own mask, only the sum
  const uint32_t v0 = (y0 + n0 - 1u) & mx;
  const uint32_t v1 = (0u - y1 - n1) & mx;
#if BC_ALU_ADDS
  if (!kWide) {
    // the same steps 5-9 with every sum in three-input form (p < 2^31, so
    // every sum below stays under 2^32; a value in [0, 2p) reduces to the
    // minimum of itself and itself minus p, which wraps above it when < p)
    const uint32_t z1 = k.zero1, z2 = k.zero2, negp = k.neg_p;
    // step 5: m0 = v0, or 2^lx (< p) when v0 = 0, as ((v0 - 1) mod 2^lx) + 1
    // with v0 - 1 taken straight from the window sum (no compare and select)
    const uint32_t m0 = ((y0 + n0 - 2u) & mx) + 1u + z1;
    const uint32_t m1 = v1 + k.p_minus_2lx + z1;
    const uint32_t rho = mulhi_64x32<1>(rz.x, rz.y, k.mp.pm1);   // 1 + floor(w (p - 1) / 2^64)
    const uint32_t zk = mulhi_64x32(rz.z, rz.w, p);
    const uint32_t q0 = mont_mul_raw(m0, rho, k.mp), q1 = mont_mul_raw(m1, rho, k.mp);
    const uint32_t u0 = min(q0, q0 + negp + z1);
    const uint32_t u1 = min(q1, q1 + negp + z2);
    const uint32_t a0 = u0 + zk + z1;                  // step 8: P0 adds z_k
    w0 = min(a0, a0 + negp + z2);
    const uint32_t a1 = u1 - zk + z1;                  // P1 subtracts it
    w1 = min(a1, a1 + p + z2);
    const uint32_t s = w0 + w1 + z1;                   // step 9: below 2p
    return min(s, s + negp + z2);                      // s mod p: 0 iff s is 0 or p
  }
#endif
  // step 5: Alg. modswitch
  const uint32_t m0 = v0 ? v0 : k.two_lx;
  const uint32_t m1 = v1 + k.p_minus_2lx;
  // step 7: rho_k, z_k from the slot's seed01 block rz; the mask r_k =
  // rho_k 2^-32 mod p, so one Montgomery product m rho 2^-32 is m r_k
  const uint32_t rho = mulhi_64x32<1>(rz.x, rz.y, k.mp.pm1);
  const uint32_t z = mulhi_64x32(rz.z, rz.w, p);
  w0 = mont_mul<kWide>(m0, rho, k.mp);
  w1 = mont_mul<kWide>(m1, rho, k.mp);
  // step 8: reshare (P0 adds z_k, P1 subtracts it) and send to P2
  w0 = M::add(w0, z, p);
  w1 = M::sub(w1, z, p);
  // step 9: P2 reconstructs w_k
  return M::add(w0, w1, p);
}

// The same slot from the flipped share and 2^l minus the other flipped share,
// f0c and nf1c, already shifted right by the key offset c (once per element),
// so the window of index i starts at bit i.
template <int LX, bool SHORT, typename Lane>
__device__ __forceinline__ uint32_t slot_reconstruct(const ReluConsts& k, Lane f0c, Lane nf1c,
                                                     uint32_t i, const U32x4& rz, uint32_t& w0,
                                                     uint32_t& w1) {
  const uint32_t lx = LX ? (uint32_t)LX : k.lx;
  return slot_from_windows<LX>(k, window32<SHORT>(f0c, i), window32<SHORT>(nf1c, i),
                               (i < lx) ? 1u : 33u, rz, w0, w1);
}

// The same slot with P2's zero test: 1 when w_k = 0.
template <int LX, bool SHORT, typename Lane>
__device__ __forceinline__ uint32_t slot_zero_test(const ReluConsts& k, Lane f0c, Lane nf1c,
                                                   uint32_t i, const U32x4& rz, uint32_t& w0,
                                                   uint32_t& w1) {
  return slot_reconstruct<LX, SHORT>(k, f0c, nf1c, i, rz, w0, w1) == 0u ? 1u : 0u;
}

// Steps 1-9 of one element, shuffle first: the seed01 stream gives t and
// the Fisher-Yates shuffle of the lx + 1 slots, then every message slot k
// runs steps 3-9 on the window index perm[k].  Returns DReLU' (1 if some
// w_k is zero); t is the flip bit.
template <typename Lane, int LX, bool SHORT, bool AUDIT, int UNROLL>
__device__ __forceinline__ uint32_t slots_after_shuffle(const ReluConsts& k, const RoundKeys& rk,
                                                        const ElemPhilox& ep, Lane s0, Lane s1,
                                                        uint32_t* perm, const AuditPtrs& aud,
                                                        uint64_t out_idx, const uint64_t* r2tab,
                                                        uint32_t& t_out) {
  const uint32_t lx = LX ? (uint32_t)LX : k.lx;
  const uint32_t L = lx + 1;
  const Lane mask = (Lane)k.ring_mask;
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
    const uint64_t mbp = (uint64_t)kPhiloxM1 * b;
    const U32x4 wb = r2tab ? perm_stream.block_p0(mbp, r2tab[b], rk) : perm_stream.block(mbp, rk);
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
  // (both shifted right by the key offset c for the windows of step 3)
  const Lane f0 = (t ? ring_neg(s0, mask) : s0) >> k.c;
  const Lane nf1 = (t ? s1 : ring_neg(s1, mask)) >> k.c;   // 2^l - [x]_1 of the flipped share

  // ---- steps 3-9 over message slots k ----------------------------------------
  uint32_t any_zero = 0;
  const StreamPhilox mask_stream(ep, kPair01, kPurMask, rk);
  uint64_t mb = 0;   // M1 * slot, the round-1 product of the slot's mask block
  constexpr int kUnroll = UNROLL > 0 ? UNROLL : (LX ? LX + 1 : 2);
#pragma unroll kUnroll
  for (uint32_t slot = 0; slot < L; ++slot, mb += kPhiloxM1) {
    uint32_t w0, w1;
    const U32x4 rz =
        r2tab ? mask_stream.block_p0(mb, r2tab[slot], rk) : mask_stream.block(mb, rk);
    any_zero |= slot_zero_test<LX, SHORT>(k, f0, nf1, perm[slot * kBlock], rz, w0, w1);
    if (AUDIT) {
      if (aud.w0) aud.w0[out_idx * L + slot] = w0;
      if (aud.w1) aud.w1[out_idx * L + slot] = w1;
    }
  }
  t_out = t;
  return any_zero;
}

// The same steps with the shuffle and the slots interleaved (fixed key width
// only): Fisher-Yates from the top leaves position j final once step j has
// run, so slot j's message follows its shuffle step directly, with window
// index the value just swapped into position j; the slots are taken in the
// order lx, ..., 1, 0, and their zero tests are OR-ed as before.
template <typename Lane, int LX, bool SHORT, bool AUDIT>
__device__ __forceinline__ uint32_t slots_with_shuffle(const ReluConsts& k, const RoundKeys& rk,
                                                       const ElemPhilox& ep, Lane s0, Lane s1,
                                                       uint32_t* perm, const AuditPtrs& aud,
                                                       uint64_t out_idx, const uint64_t* r2tab,
                                                       uint32_t& t_out) {
  constexpr uint32_t L = LX + 1;
  const Lane mask = (Lane)k.ring_mask;
#pragma unroll
  for (uint32_t s = 0; s < L; ++s) perm[s * kBlock] = s;
  const StreamPhilox perm_stream(ep, kPair01, kPurPerm, rk);
  const StreamPhilox mask_stream(ep, kPair01, kPurMask, rk);
  uint32_t t = 0, any_zero = 0;
  Lane f0 = s0, nf1 = s1;
#pragma unroll
  for (uint32_t b = 0; b < (L + 3) / 4; ++b) {
    const uint64_t mbp = (uint64_t)kPhiloxM1 * b;
    const U32x4 wb = r2tab ? perm_stream.block_p0(mbp, r2tab[b], rk) : perm_stream.block(mbp, rk);
    const uint32_t ws[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t widx = 4 * b + q;
      if (widx == 0) {
        t = ws[0] & 1u;                                   // steps 1-2
        f0 = (t ? ring_neg(s0, mask) : s0) >> k.c;        // shifted by c for step 3
        nf1 = (t ? s1 : ring_neg(s1, mask)) >> k.c;
      } else if (widx < L) {
        const uint32_t j = L - widx;                      // step 6, then slot j
        const uint32_t partner = __umulhi(ws[q], j + 1);
        const uint32_t a = perm[j * kBlock];
        const uint32_t c = perm[partner * kBlock];
        // the swap's other half, perm[j] = c, is not stored: position j is
        // final and later steps (partners <= j - 1) never read it
        perm[partner * kBlock] = a;
        const uint64_t mb = (uint64_t)kPhiloxM1 * j;
        const U32x4 rz =
            r2tab ? mask_stream.block_p0(mb, r2tab[j], rk) : mask_stream.block(mb, rk);
        uint32_t w0, w1;
        any_zero |= slot_zero_test<LX, SHORT>(k, f0, nf1, c, rz, w0, w1);
        if (AUDIT) {
          if (aud.w0) aud.w0[out_idx * L + j] = w0;
          if (aud.w1) aud.w1[out_idx * L + j] = w1;
        }
      }
    }
  }
  const U32x4 rz = r2tab ? mask_stream.block_p0(0, r2tab[0], rk) : mask_stream.block(0, rk);
  uint32_t w0, w1;
  any_zero |= slot_zero_test<LX, SHORT>(k, f0, nf1, perm[0], rz, w0, w1);   // slot 0
  if (AUDIT) {
    if (aud.w0) aud.w0[out_idx * L] = w0;
    if (aud.w1) aud.w1[out_idx * L] = w1;
  }
  t_out = t;
  return any_zero;
}

// Alg. drelu / Alg. relu for one element.  `perm` points at this thread's
// column of the shared-memory shuffle table (stride kBlock words).
// DPONLY: stop after P2's step 9 and return DReLU' in out0 and t in out1
// (the RSS protocol finishes differently).  UNROLL: unroll of the loop over
// the lx + 1 message slots (the key-bit loop); 0 = all of it for a fixed LX,
// 2 otherwise.  r2tab (optional): the CTA's
// table of round2_product(tensor_id, b) for b = 0 .. lx, shared by its threads.
template <typename Lane, int LX, bool SHORT, bool RELU, bool AUDIT, bool DPONLY = false,
          int UNROLL = kSlotUnroll>
__device__ __forceinline__ void bicoptor_element(const ReluConsts& k, const RoundKeys& rk,
                                                 uint32_t tensor_id, Lane s0, Lane s1,
                                                 uint64_t elem, uint32_t* perm, Lane& out0,
                                                 Lane& out1, const AuditPtrs& aud,
                                                 uint64_t out_idx,
                                                 const uint64_t* r2tab = nullptr) {
  const Lane mask = (Lane)k.ring_mask;
  const ElemPhilox ep(elem, tensor_id);

  uint32_t t;
  const uint32_t any_zero =
      (BC_INTERLEAVE && LX)
          ? slots_with_shuffle<Lane, (LX ? LX : 1), SHORT, AUDIT>(k, rk, ep, s0, s1, perm, aud,
                                                                  out_idx, r2tab, t)
          : slots_after_shuffle<Lane, LX, SHORT, AUDIT, UNROLL>(k, rk, ep, s0, s1, perm, aud,
                                                                out_idx, r2tab, t);
  const uint32_t dprime = any_zero;
  if (DPONLY) {
    out0 = (Lane)dprime;
    out1 = (Lane)t;
    return;
  }

  if (!RELU) {
    // step 10: [DReLU']_0 = d0 from seed02 (P0 derives it), [DReLU']_1 to P1
    const U32x4 rb = ep.block_tab(kPair02, kPurReply, 0, r2tab, rk);
    const Lane d0 = block_elem<Lane>(rb, 0) & mask;
    const Lane d1 = ((Lane)dprime - d0) & mask;
    // step 11: [DReLU] = [DReLU' xor t], the public t added by P0
    out0 = t ? (Lane)((Lane)1 - d0) & mask : d0;
    out1 = t ? ring_neg(d1, mask) : d1;
    if (AUDIT && aud.reply) store_lane<Lane>(aud.reply, out_idx, d1);
  } else {
    const Triple<Lane> T = draw_triple<Lane>(ep, kPurReluTriple, mask, rk, r2tab);
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

}  // namespace bc
