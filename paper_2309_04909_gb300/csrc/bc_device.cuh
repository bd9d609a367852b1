// Device building blocks of the Bicoptor 2.0 hot path (sm_103a).
//
// Integer-only: ring arithmetic in Z_{2^l} on uint32/uint64 lanes, Z_p
// arithmetic for the masked messages (p < 2^32) by Montgomery multiplication
// (P. L. Montgomery, "Modular multiplication without trial division", Math.
// Comp. 1985), and the counter-based Philox-4x32-10 generator (Salmon et al.,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011) that expands the
// pre-shared seeds of Sec. 2.1 inside registers.
#pragma once
#include <stdint.h>

namespace bc {

// ---------------------------------------------------------------------------
// Philox-4x32-10.  The ten round keys are precomputed on the host and passed
// in kernel parameters, so each round is two 32x32->64 multiplies and two
// three-input XORs, with the key read straight from the constant bank.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

struct U32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return U32x4{c0, c1, c2, c3};
}

// Rounds 2..10 of Philox-4x32-10 (round 1 done by the caller).
__device__ __forceinline__ U32x4 philox_rounds_2_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                    uint32_t c3, const RoundKeys& rk) {
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return U32x4{c0, c1, c2, c3};
}

// Rounds 3..10 of Philox-4x32-10 (rounds 1 and 2 done by the caller).
__device__ __forceinline__ U32x4 philox_rounds_3_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                    uint32_t c3, const RoundKeys& rk) {
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return U32x4{c0, c1, c2, c3};
}

// Stream tags: which pre-shared seed a draw belongs to, and what it is for.
// counter = (lo32(elem), tensor_id, block, pair << 24 | purpose << 16 | elem >> 32)
enum : uint32_t {
  kPair01 = 0x01, kPair02 = 0x02, kPair12 = 0x12, kPairDealer = 0xDE,
  kPair012 = 0x03,   // seed012, all three parties (RSS)
  kPair2 = 0x20      // seed2, P2 alone (RSS)
};
enum : uint32_t {
  kPurShare = 1,        // dealer: R of the 2-of-2 sharing
  kPurPerm = 2,         // seed01: flip bit t and the shuffle words
  kPurMask = 3,         // seed01: (r_k, z_k) of message slot k, block k
  kPurReply = 4,        // seed02: P0's share of DReLU'
  kPurReluTriple = 5,   // seed02: a0,b0,c0 / seed12: a1,b1 of the ReLU product
  kPurMulTriple = 6,    // seed02: a0,b0,c0 / seed12: a1,b1 of a Beaver product
  kPurAby3 = 7,         // seed02: [r]_0, [r']_0 / seed12: [r]_1 of ABY3 truncation
  kPurRssT = 8,         // seed012: alpha_0..2, the sharing of t (RSS)
  kPurRssS = 9,         // seed2: s / seed012: [s]_1 / seed12: [s]_2 (RSS)
  kPurRssZ = 10,        // seed012: zero sharing of [s][t] (RSS)
  kPurRssZr = 11,       // seed012: zero sharing of the RSS ReLU product
  kPurB1Mask = 12,      // seed01: (r_k, z_k) of slot k, the Bicoptor 1.0-style protocol
};

__device__ __forceinline__ uint32_t stream_tag(uint32_t pair, uint32_t purpose, uint64_t elem) {
  return (pair << 24) | (purpose << 16) | (uint32_t)((elem >> 32) & 0xffffu);
}

__device__ __forceinline__ U32x4 draw_block(uint32_t pair, uint32_t purpose, uint32_t tensor_id,
                                            uint64_t elem, uint32_t block, const RoundKeys& rk) {
  return philox((uint32_t)elem, tensor_id, block, stream_tag(pair, purpose, elem), rk);
}

// Round 2's first product of block b of any stream: M0 * (hi32(M1 b) ^
// tensor_id ^ k0[0]).  Its operand is round 1's output word 0, which depends
// on the block index and the tensor id only -- not on the element or the
// stream -- so a CTA working on one tensor can share a table of it.
__host__ __device__ __forceinline__ uint64_t round2_product(uint32_t tensor_id, uint32_t b,
                                                            const RoundKeys& rk) {
  const uint32_t a0 = (uint32_t)(((uint64_t)kPhiloxM1 * b) >> 32) ^ tensor_id ^ rk.k0[0];
  return (uint64_t)kPhiloxM0 * a0;
}

// Philox blocks of one element with round 1 factored: every block of the
// element shares c0 = lo32(elem), so M0 * c0 is computed once per element;
// M1 * c2 (c2 = block index) is a constant or a running sum in the caller.
struct ElemPhilox {
  uint32_t e_hi, e_lo;    // M0 * lo32(elem)
  uint32_t elem_hi16;     // (elem >> 32) & 0xffff
  uint32_t tensor_id;
  __device__ __forceinline__ ElemPhilox(uint64_t elem, uint32_t tid) {
    const uint64_t pe = (uint64_t)kPhiloxM0 * (uint32_t)elem;
    e_hi = (uint32_t)(pe >> 32);
    e_lo = (uint32_t)pe;
    elem_hi16 = (uint32_t)((elem >> 32) & 0xffffu);
    tensor_id = tid;
  }
  // block with M1 * block = mb (64-bit)
  __device__ __forceinline__ U32x4 block(uint32_t pair, uint32_t purpose, uint64_t mb,
                                         const RoundKeys& rk) const {
    const uint32_t tag = (pair << 24) | (purpose << 16) | elem_hi16;
    return philox_rounds_2_10((uint32_t)(mb >> 32) ^ tensor_id ^ rk.k0[0], (uint32_t)mb,
                              e_hi ^ tag ^ rk.k1[0], e_lo, rk);
  }
  __device__ __forceinline__ U32x4 block_at(uint32_t pair, uint32_t purpose, uint32_t b,
                                            const RoundKeys& rk) const {
    return block(pair, purpose, (uint64_t)kPhiloxM1 * b, rk);
  }
  // block b with round 2's first product p0 = round2_product(tensor_id, b)
  // supplied by the caller
  __device__ __forceinline__ U32x4 block_p0(uint32_t pair, uint32_t purpose, uint32_t b,
                                            uint64_t p0, const RoundKeys& rk) const {
    const uint32_t tag = (pair << 24) | (purpose << 16) | elem_hi16;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * (e_hi ^ tag ^ rk.k1[0]);
    const uint32_t x1 = (uint32_t)((uint64_t)kPhiloxM1 * b);   // round 1's word 1
    return philox_rounds_3_10((uint32_t)(p1 >> 32) ^ x1 ^ rk.k0[1], (uint32_t)p1,
                              (uint32_t)(p0 >> 32) ^ e_lo ^ rk.k1[1], (uint32_t)p0, rk);
  }
  // block_at, or block_p0 from the table r2 (r2[b] = round2_product(tensor_id, b))
  __device__ __forceinline__ U32x4 block_tab(uint32_t pair, uint32_t purpose, uint32_t b,
                                             const uint64_t* r2, const RoundKeys& rk) const {
    return r2 ? block_p0(pair, purpose, b, r2[b], rk) : block_at(pair, purpose, b, rk);
  }
};

// The blocks of one (element, pair, purpose) stream, e.g. the lx + 1 mask
// blocks of an element: after round 1 their counter words 2 and 3 do not
// depend on the block index, so round 2's product M1 * word2 is the same for
// all of them and is computed once here.
struct StreamPhilox {
  uint32_t q_hi, q_lo;    // round 2: M1 * (hi32(M0 lo32(elem)) ^ tag ^ k1[0])
  uint32_t e_lo;          // lo32(M0 lo32(elem)), word 3 after round 1
  uint32_t tensor_id;
  __device__ __forceinline__ StreamPhilox(const ElemPhilox& ep, uint32_t pair, uint32_t purpose,
                                          const RoundKeys& rk) {
    const uint32_t tag = (pair << 24) | (purpose << 16) | ep.elem_hi16;
    const uint64_t q = (uint64_t)kPhiloxM1 * (ep.e_hi ^ tag ^ rk.k1[0]);
    q_hi = (uint32_t)(q >> 32);
    q_lo = (uint32_t)q;
    e_lo = ep.e_lo;
    tensor_id = ep.tensor_id;
  }
  // block with M1 * block = mb (64-bit); equal to ElemPhilox::block
  __device__ __forceinline__ U32x4 block(uint64_t mb, const RoundKeys& rk) const {
    const uint32_t a0 = (uint32_t)(mb >> 32) ^ tensor_id ^ rk.k0[0];
    return block_p0(mb, (uint64_t)kPhiloxM0 * a0, rk);
  }
  // the same with round 2's first product p0 = round2_product(tensor_id, block)
  __device__ __forceinline__ U32x4 block_p0(uint64_t mb, uint64_t p0, const RoundKeys& rk) const {
    return philox_rounds_3_10(q_hi ^ (uint32_t)mb ^ rk.k0[1], q_lo,
                              (uint32_t)(p0 >> 32) ^ e_lo ^ rk.k1[1], (uint32_t)p0, rk);
  }
};

// ---------------------------------------------------------------------------
// Ring Z_{2^l} on lanes.  Lane = uint32_t for l <= 32, uint64_t for l <= 64.
// ---------------------------------------------------------------------------
template <typename Lane>
__device__ __forceinline__ Lane ring_neg(Lane a, Lane mask) {
  return (Lane)(Lane(0) - a) & mask;
}

// The j-th ring element of a block (0 <= j < 4 for 32-bit lanes, 0 <= j < 2
// for 64-bit lanes; 64-bit elements take two words, low word first).
template <typename Lane>
__device__ __forceinline__ Lane block_elem(const U32x4& b, int j);
template <>
__device__ __forceinline__ uint32_t block_elem<uint32_t>(const U32x4& b, int j) {
  return j == 0 ? b.x : j == 1 ? b.y : j == 2 ? b.z : b.w;
}
template <>
__device__ __forceinline__ uint64_t block_elem<uint64_t>(const U32x4& b, int j) {
  return j == 0 ? ((uint64_t)b.y << 32 | b.x) : ((uint64_t)b.w << 32 | b.z);
}

// Beaver product of one element (Sec. 2.2, the multiplication of the linear
// layers): the triple a0, b0, c0 comes from seed02 and a1, b1 from seed12
// (purpose kPurMulTriple), P2 completes it with c1 = (a0 + a1)(b0 + b1) - c0;
// P0 and P1 open d = x - a and e = y - b, and P0 adds the public d e.
// r2 (optional): round2_product(tensor_id, b) for b = 0, 1.
template <typename Lane>
__device__ __forceinline__ void beaver_mul(const ElemPhilox& ep, const RoundKeys& rk, Lane mask,
                                           Lane x0, Lane x1, Lane y0, Lane y1, Lane& o0,
                                           Lane& o1, const uint64_t* r2 = nullptr) {
  const U32x4 q0 = ep.block_tab(kPair02, kPurMulTriple, 0, r2, rk);
  const U32x4 q1 = ep.block_tab(kPair12, kPurMulTriple, 0, r2, rk);
  Lane a0, b0, c0;
  if (sizeof(Lane) == 4) {
    a0 = (Lane)q0.x; b0 = (Lane)q0.y; c0 = (Lane)q0.z;
  } else {
    const U32x4 q2 = ep.block_tab(kPair02, kPurMulTriple, 1, r2, rk);
    a0 = block_elem<Lane>(q0, 0); b0 = block_elem<Lane>(q0, 1); c0 = block_elem<Lane>(q2, 0);
  }
  const Lane a1 = block_elem<Lane>(q1, 0) & mask, b1 = block_elem<Lane>(q1, 1) & mask;
  a0 &= mask; b0 &= mask; c0 &= mask;
  const Lane c1 = (Lane)((a0 + a1) * (b0 + b1) - c0) & mask;   // P2 -> P1
  const Lane d = (Lane)((x0 - a0) + (x1 - a1)) & mask;           // opened x - a
  const Lane e = (Lane)((y0 - b0) + (y1 - b1)) & mask;           // opened y - b
  o0 = (Lane)(d * e + d * b0 + e * a0 + c0) & mask;
  o1 = (Lane)(d * b1 + e * a1 + c1) & mask;
}

// ---------------------------------------------------------------------------
// Z_p, odd p < 2^32 with p in (2^lx, 2^(lx+1)).
// ---------------------------------------------------------------------------
struct ModP {
  uint32_t p;      // the prime
  uint32_t pinv;   // -p^{-1} mod 2^32
  uint32_t r2;     // 2^64 mod p
  uint32_t pm1;    // p - 1
};

// Montgomery product a * b * 2^-32 mod p for a, b < p < 2^32.  With
// t = a b and q = -t p^-1 mod 2^32, t + q p is a multiple of 2^32 and
// (t + q p) / 2^32 < 2p, so one conditional subtraction lands in [0, p).
// t + q p < p^2 + 2^32 p exceeds 64 bits once p > 0.618 * 2^32 (possible for
// key width lx = 31), so WIDE keeps the carry out of the 64-bit sum; for
// p < 2^31 the sum always fits.
template <bool WIDE = true>
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const ModP& m) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * m.pinv;
  const uint64_t u = t + (uint64_t)q * m.p;
  const uint32_t r = (uint32_t)(u >> 32);
  const bool carry = WIDE && u < t;      // the quotient is r + 2^32
  return (carry || r >= m.p) ? r - m.p : r;
}

// The Montgomery quotient (a b + q p) / 2^32 in [0, 2p), before the final
// subtraction, for p < 2^31 (the 64-bit sum cannot overflow).
__device__ __forceinline__ uint32_t mont_mul_raw(uint32_t a, uint32_t b, const ModP& m) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * m.pinv;
  return (uint32_t)((t + (uint64_t)q * m.p) >> 32);
}

// a + b mod p and a - b mod p for a, b < p (p < 2^32 so the sum may wrap
// 32 bits only when p > 2^31; handled through 64-bit compare).
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint64_t s = (uint64_t)a + b;
  return (uint32_t)(s >= p ? s - p : s);
}
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p) {
  return a >= b ? a - b : a + (p - b);
}

// floor(w * q / 2^64) + ADD for a 64-bit w given as (hi, lo), a 32-bit q and
// a constant ADD (0 or 1; the sum must fit 32 bits): floor((hi q +
// floor(lo q / 2^32)) / 2^32) = hi32(hi q) + the carry out of lo32(hi q) +
// hi32(lo q).  The sum runs as a multiply-add carry chain (mad.lo.cc, then
// madc.hi, whose addend is ADD), not as a 64-bit multiply-add whose 32-bit
// addend would first be moved into a register pair.
template <uint32_t ADD = 0>
__device__ __forceinline__ uint32_t mulhi_64x32(uint32_t lo, uint32_t hi, uint32_t q) {
  const uint32_t a_hi = __umulhi(lo, q);
  uint32_t r;
  asm("{\n\t.reg .u32 t;\n\t"
      "mad.lo.cc.u32 t, %1, %2, %3;\n\t"
      "madc.hi.u32 %0, %1, %2, %4;\n\t}"
      : "=r"(r)
      : "r"(hi), "r"(q), "r"(a_hi), "n"(ADD));
  return r;
}

}  // namespace bc
