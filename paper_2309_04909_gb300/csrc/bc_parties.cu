// Party-separated Bicoptor 2.0 DReLU / ReLU (Alg. drelu, Alg. relu): each
// party's local computation is its own kernel, and every message between the
// parties is a device buffer written by the sender's kernel and read by the
// receiver's.  Three launches, in protocol order:
//   1. parties_local   P0 and P1 (blockIdx.y = party), each from its own share
//                      and its own expansion of the pre-shared seeds: steps 1-8,
//                      w messages to P2 bit-packed at lx+1 bits per value;
//                      ReLU: the opening [x]_j - [a]_j to the other party
//   2. helper          P2: preprocessing [c]_1 -> P1 (ReLU); step 9 on the two
//                      w messages; step 10 reply [DReLU']_1 -> P1 (DReLU) or
//                      e = DReLU' - b -> P0, P1 (ReLU)
//   3. parties_finish  P0 and P1: step 11 / the Beaver finish from the
//                      messages they received
// Unlike the fused kernel, P0 and P1 each expand seed01 (t, the shuffle, the
// masks) themselves, as separate servers would.
//
// Packed w layout: elements in groups of 32; for group g and slot k the lx+1
// words at (g * L + k) * (lx+1) (L = lx+1 slots) hold the 32 values of the
// group, element 32 g + l at bits [l (lx+1), (l+1)(lx+1)).  A group's whole
// message is thus contiguous, and so are the 8 groups of one 256-thread CTA.
// The group count is padded to a multiple of 8, so the buffer holds the
// protocol's (lx+1)^2 bits per element and sender, padded to a multiple of
// 256 elements.  P2's kernel fetches its CTA's two messages with bulk
// asynchronous copies (cp.async.bulk) into shared memory.
#include "bc_internal.h"

namespace bc {
namespace {

constexpr int kPB = kBlock;             // threads per CTA
constexpr int kWarps = kPB / 32;        // groups of 32 elements per CTA
constexpr uint32_t kBulkChunk = 16384;  // bytes per bulk copy instruction
constexpr uint64_t kWaitNs = 50000000;  // P2's wait for its messages: 50 ms
constexpr uint64_t kTestWaitNs = 1000000;

// ---- bulk asynchronous copies and their mbarrier ----------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// make the initialised barrier visible to the async proxy that completes it
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) that completes its bytes on the mbarrier at `bar`
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0u;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier for at most limit_ns nanoseconds
// (and at most 2^22 polls); false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

template <typename Lane>
__device__ __forceinline__ Lane lane_at(const void* p, uint64_t i) {
  return static_cast<const Lane*>(p)[i];
}
template <typename Lane>
__device__ __forceinline__ void lane_put(void* p, uint64_t i, Lane v) {
  static_cast<Lane*>(p)[i] = v;
}

// seed01: t and the Fisher-Yates shuffle (steps 1 and 6), into `perm`
// (this thread's column of the shared table, stride kPB).
__device__ __forceinline__ uint32_t seed01_shuffle(const ElemPhilox& ep, uint32_t L,
                                                   uint32_t* perm, const RoundKeys& rk,
                                                   const uint64_t* r2) {
  for (uint32_t s = 0; s < L; ++s) perm[s * kPB] = s;
  uint32_t t = 0;
  const uint32_t nblk = (L + 3) >> 2;
  const StreamPhilox stream(ep, kPair01, kPurPerm, rk);
  for (uint32_t b = 0; b < nblk; ++b) {
    const U32x4 wb = stream.block_p0((uint64_t)kPhiloxM1 * b, r2[b], rk);
    const uint32_t ws[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t widx = 4 * b + q;
      if (widx == 0) {
        t = ws[0] & 1u;
      } else if (widx < L) {
        const uint32_t j = L - widx;
        const uint32_t partner = __umulhi(ws[q], j + 1);
        const uint32_t a = perm[j * kPB];
        const uint32_t c = perm[partner * kPB];
        perm[j * kPB] = c;
        perm[partner * kPB] = a;
      }
    }
  }
  return t;
}

__device__ __forceinline__ uint32_t seed01_t(const ElemPhilox& ep, const RoundKeys& rk,
                                             const uint64_t* r2) {
  return ep.block_tab(kPair01, kPurPerm, 0, r2, rk).x & 1u;
}

// The CTA's table of round2_product(tensor_id, b), b < kMaxSlots (one
// widening product less per Philox block of every element); call from all
// threads before any returns.
__device__ __forceinline__ void fill_round2(uint64_t* r2, uint32_t tensor_id,
                                            const RoundKeys& rk) {
  if (threadIdx.x < kMaxSlots) r2[threadIdx.x] = round2_product(tensor_id, threadIdx.x, rk);
  __syncthreads();
}

// Pack the group's L slots after the slot loop.  `vals` holds the warp's
// values, value of lane l for slot k at vals[k * kPB + l] (each thread's
// column of the shuffle table, overwritten slot by slot).  Lane j < B writes
// word j of every slot: bits [32 j, 32 j + 32) of the 32 B-bit values laid end
// to end.  Value l0 = floor(32 j / B) enters shifted right by r0 = 32 j - l0 B,
// the next ones shifted left by B - r0, 2B - r0, ...  For B >= 16 a word takes
// at most three values, and the shifts are fixed before the slot loop.
__device__ __forceinline__ void pack_group(const uint32_t* vals, uint32_t L, uint32_t B,
                                           uint32_t lane, uint32_t* dst) {
  if (lane >= B) return;
  const uint32_t lo_bit = lane * 32u;
  const uint32_t l0 = lo_bit / B;
  const uint32_t r0 = lo_bit - l0 * B;
  if (B >= 16u) {
    const uint32_t s1 = B - r0, s2 = s1 + B;                  // 0 < s1 <= B
    const bool has1 = l0 + 1u <= 31u && s1 < 32u;
    const bool has2 = l0 + 2u <= 31u && s2 < 32u;
    const uint32_t* v0 = vals + l0;
    const uint32_t* v1 = vals + (has1 ? l0 + 1u : l0);
    const uint32_t* v2 = vals + (has2 ? l0 + 2u : l0);
    const uint32_t m1 = has1 ? 0xffffffffu : 0u, m2 = has2 ? 0xffffffffu : 0u;
    const uint32_t t1 = has1 ? s1 : 0u, t2 = has2 ? s2 : 0u;
    for (uint32_t slot = 0; slot < L; ++slot) {
      const uint32_t o = slot * kPB;
      dst[slot * B] = (v0[o] >> r0) | ((v1[o] << t1) & m1) | ((v2[o] << t2) & m2);
    }
    return;
  }
  const uint32_t l1 = min(31u, (lo_bit + 31u) / B);
  for (uint32_t slot = 0; slot < L; ++slot) {
    uint32_t word = vals[slot * kPB + l0] >> r0;
    for (uint32_t l = l0 + 1u, sh = B - r0; l <= l1; ++l, sh += B)   // sh < 32
      word |= vals[slot * kPB + l] << sh;
    dst[slot * B] = word;
  }
}

constexpr uint32_t kBothParties = 0xffffffffu;   // PartyArgs::party0: P0 and P1 in one launch

struct PartyArgs {
  ReluConsts k;
  const void* sh[2];        // [x]_0 (P0's input), [x]_1 (P1's input)
  void* out[2];             // output shares of P0, P1
  uint32_t* w[2];           // P0 -> P2, P1 -> P2 packed messages
  void* open[2];            // P0 -> P1, P1 -> P0 openings (ReLU)
  void* reply;              // P2 -> P1 / P2 -> P0, P1
  void* pre_c1;             // P2 -> P1 preprocessing (ReLU)
  uint64_t n;
  int* status;              // set to BC_ETIMEOUT if P2 gives up waiting
  uint32_t drop_copies;     // test hook: P2 issues no copies, so its wait runs out
  uint64_t wait_ns;         // P2's wait limit
  uint32_t party0;          // launches 1 and 3: party of blockIdx.y = 0 (grid y = 2 - party0
                            // for both parties from 0, 1 for one party alone)
};

// ---- launch 1: P0 and P1, steps 1-8 (+ opening of x - a) --------------------
template <typename Lane, bool RELU>
__global__ void __launch_bounds__(kPB)
    parties_local_kernel(const PartyArgs a) {
  __shared__ uint32_t perm_s[kMaxSlots * kPB];
  __shared__ uint64_t r2_s[kMaxSlots];
  fill_round2(r2_s, a.k.tensor_id, a.k.rk);
  const uint32_t party = a.party0 + blockIdx.y;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t i = (uint64_t)blockIdx.x * kPB + threadIdx.x;
  const bool valid = i < a.n;
  // a warp past the end owns no group: it must not pack (the group index of
  // every lane is its warp's, so a partial warp packs its own group only)
  if (!__any_sync(0xffffffffu, valid)) return;
  const uint64_t g = ((uint64_t)blockIdx.x * kPB + warp * 32u) >> 5;
  const ReluConsts& k = a.k;
  const uint32_t lx = k.lx, L = lx + 1, B = lx + 1;
  const Lane mask = (Lane)k.ring_mask;
  const uint64_t elem = k.elem_base + (valid ? i : 0);
  const ElemPhilox ep(elem, k.tensor_id);
  uint32_t* perm = perm_s + threadIdx.x;
  const uint32_t t = seed01_shuffle(ep, L, perm, k.rk, r2_s);
  const Lane s = valid ? lane_at<Lane>(a.sh[party], i) : (Lane)0;
  // steps 1-2 and the P1 pre-negation: P0 keeps [x]_0 (flipped), P1 keeps
  // 2^l - [x]_1 of its flipped share
  // (shifted right by the key offset c once, so window i starts at bit i)
  const Lane f =
      (party == 0 ? (t ? ring_neg(s, mask) : s) : (t ? s : ring_neg(s, mask))) >> k.c;
  const StreamPhilox mask_stream(ep, kPair01, kPurMask, k.rk);
  uint64_t mb = 0;
  for (uint32_t slot = 0; slot < L; ++slot, mb += kPhiloxM1) {
    const uint32_t ii = perm[slot * kPB];
    const uint32_t y = (uint32_t)((uint64_t)f >> ii);
    // u_(i+1): y shifted by one, or 0 for i = lx (u_(lx+1) := 0) by a shift
    // clamped at 32; the sums mod 2^lx need no mask on their terms
    const uint32_t n = __funnelshift_rc(y, 0u, (ii < lx) ? 1u : 33u);
    uint32_t m;
    if (party == 0) {
      // steps 3-5: v = u_i + u_(i+1) - 1, and 2^lx in place of v = 0, as
      // ((v - 1) mod 2^lx) + 1
      m = ((y + n - 2u) & k.mx) + 1u;
    } else {
      m = ((0u - y - n) & k.mx) + k.p_minus_2lx;
    }
    const U32x4 rz = mask_stream.block_p0(mb, r2_s[slot], k.rk);              // step 7
    const uint32_t rho = mulhi_64x32<1>(rz.x, rz.y, k.mp.pm1);
    const uint32_t z = mulhi_64x32(rz.z, rz.w, k.mp.p);
    uint32_t w = mont_mul(m, rho, k.mp);
    w = party == 0 ? add_mod(w, z, k.mp.p) : sub_mod(w, z, k.mp.p);          // step 8
    perm[slot * kPB] = valid ? w : 0u;   // the table entry read above is not needed again
  }
  __syncwarp();
  pack_group(perm_s + warp * 32u, L, B, lane, a.w[party] + g * L * B + lane);
  if (RELU && valid) {
    // opening of d = x - a: P0 draws a0 from seed02, P1 draws a1 from seed12
    const U32x4 q = ep.block_tab(party == 0 ? kPair02 : kPair12, kPurReluTriple, 0, r2_s, k.rk);
    const Lane ai = block_elem<Lane>(q, 0) & mask;
    lane_put<Lane>(a.open[party], i, (Lane)(s - ai) & mask);
  }
}

// ---- launch 2: P2 ---------------------------------------------------------------
// One thread issues bulk copies of the CTA's two messages (8 groups x L slots x
// B words from each of P0 and P1, contiguous in the group-major layout) into
// shared memory; every thread draws its element's triple from seed02 / seed12
// while they arrive, then waits on the mbarrier (bounded) and unpacks its lx+1
// value pairs from shared memory.
template <typename Lane, bool RELU>
__global__ void __launch_bounds__(kPB)
    helper_kernel(const PartyArgs a) {
  extern __shared__ __align__(128) uint32_t msg_s[];   // [2][kWarps * L * B]
  __shared__ __align__(8) uint64_t bar_s;
  __shared__ uint64_t r2_s[2];
  const ReluConsts& k = a.k;
  const uint32_t L = k.lx + 1, B = k.lx + 1;
  const uint32_t group_words = L * B;
  const uint32_t cta_words = kWarps * group_words;
  const uint32_t bar = smem_addr(&bar_s);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (threadIdx.x < 2) r2_s[threadIdx.x] = round2_product(k.tensor_id, threadIdx.x, k.rk);
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = cta_words * 4u;            // 32 L B: a multiple of 16
    mbar_arrive_expect_tx(bar, 2u * bytes);
    if (!a.drop_copies) {
      for (uint32_t party = 0; party < 2; ++party) {
        const char* src = reinterpret_cast<const char*>(a.w[party] +
                                                        (uint64_t)blockIdx.x * cta_words);
        const uint32_t dst = smem_addr(msg_s + party * cta_words);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk)
          bulk_copy_g2s(dst + off, src + off, min(kBulkChunk, bytes - off), bar);
      }
    }
  }
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t i = (uint64_t)blockIdx.x * kPB + threadIdx.x;
  const bool valid = i < a.n;
  const Lane mask = (Lane)k.ring_mask;
  const ElemPhilox ep(k.elem_base + (valid ? i : 0), k.tensor_id);
  Lane d0 = 0, a0 = 0, b0 = 0, c0 = 0, a1 = 0, b1 = 0;
  if (valid) {
    if (!RELU) {
      d0 = block_elem<Lane>(ep.block_tab(kPair02, kPurReply, 0, r2_s, k.rk), 0) & mask;
    } else {
      // P2 knows seed02 and seed12: the whole triple
      const U32x4 q0 = ep.block_tab(kPair02, kPurReluTriple, 0, r2_s, k.rk);
      const U32x4 q1 = ep.block_tab(kPair12, kPurReluTriple, 0, r2_s, k.rk);
      if (sizeof(Lane) == 4) {
        a0 = (Lane)q0.x; b0 = (Lane)q0.y; c0 = (Lane)q0.z;
      } else {
        const U32x4 q2 = ep.block_tab(kPair02, kPurReluTriple, 1, r2_s, k.rk);
        a0 = block_elem<Lane>(q0, 0); b0 = block_elem<Lane>(q0, 1);
        c0 = block_elem<Lane>(q2, 0);
      }
      a0 &= mask; b0 &= mask; c0 &= mask;
      a1 = block_elem<Lane>(q1, 0) & mask;
      b1 = block_elem<Lane>(q1, 1) & mask;
    }
  }
  if (!mbar_wait_bounded(bar, 0, a.wait_ns)) {
    // give up: report, let any copy still in flight land before the CTA's
    // shared memory is released (bounded too), and write nothing
    atomicExch(a.status, BC_ETIMEOUT);
    mbar_wait_bounded(bar, 0, a.wait_ns);
    return;
  }
  if (!valid) return;
  // this lane's B-bit field in each slot's B words: bits [sh, sh + B) of the
  // word pair (wl, wh); wh is clamped into the slot, where it is not needed
  const uint32_t bit = lane * B, wl = bit >> 5, sh = bit & 31u;
  const uint32_t wh = min(wl + 1u, B - 1u);
  const uint32_t vmask = B >= 32u ? 0xffffffffu : ((1u << B) - 1u);
  const uint32_t p = k.mp.p;
  const uint32_t* m0 = msg_s + warp * group_words;
  const uint32_t* m1 = m0 + cta_words;
  uint32_t any_zero = 0;
#pragma unroll 5
  for (uint32_t slot = 0; slot < L; ++slot, m0 += B, m1 += B) {   // step 9
    const uint32_t w0 = __funnelshift_r(m0[wl], m0[wh], sh) & vmask;
    const uint32_t w1 = __funnelshift_r(m1[wl], m1[wh], sh) & vmask;
    // w0, w1 < p, so w0 + w1 = 0 mod p iff the sum is 0 or p; as p < 2^32 a
    // 32-bit sum equals p only when the sum is p
    any_zero |= ((w0 + w1 == p) | ((w0 | w1) == 0u)) ? 1u : 0u;
  }
  if (!RELU) {
    lane_put<Lane>(a.reply, i, (Lane)((Lane)any_zero - d0) & mask);        // step 10 -> P1
    return;
  }
  lane_put<Lane>(a.pre_c1, i, (Lane)((a0 + a1) * (b0 + b1) - c0) & mask);  // [c]_1 -> P1
  lane_put<Lane>(a.reply, i, (Lane)((Lane)any_zero - b0 - b1) & mask);     // e -> P0, P1
}

// ---- launch 3: P0 and P1 finish --------------------------------------------
template <typename Lane, bool RELU>
__global__ void __launch_bounds__(kPB)
    parties_finish_kernel(const PartyArgs a) {
  __shared__ uint64_t r2_s[2];
  if (threadIdx.x < 2) r2_s[threadIdx.x] = round2_product(a.k.tensor_id, threadIdx.x, a.k.rk);
  __syncthreads();
  const uint32_t party = a.party0 + blockIdx.y;
  const uint64_t i = (uint64_t)blockIdx.x * kPB + threadIdx.x;
  if (i >= a.n) return;
  const ReluConsts& k = a.k;
  const Lane mask = (Lane)k.ring_mask;
  const ElemPhilox ep(k.elem_base + i, k.tensor_id);
  const Lane t = (Lane)seed01_t(ep, k.rk, r2_s);
  if (!RELU) {
    // step 11: P0 has d0 from seed02, P1 the reply [DReLU']_1
    if (party == 0) {
      const Lane d0 = block_elem<Lane>(ep.block_tab(kPair02, kPurReply, 0, r2_s, k.rk), 0) & mask;
      lane_put<Lane>(a.out[0], i, t ? (Lane)((Lane)1 - d0) & mask : d0);
    } else {
      const Lane d1 = lane_at<Lane>(a.reply, i);
      lane_put<Lane>(a.out[1], i, t ? ring_neg(d1, mask) : d1);
    }
    return;
  }
  const Lane e = lane_at<Lane>(a.reply, i);
  const Lane d = (Lane)(lane_at<Lane>(a.open[0], i) + lane_at<Lane>(a.open[1], i)) & mask;
  const Lane s = lane_at<Lane>(a.sh[party], i);
  Lane xd;
  if (party == 0) {
    const U32x4 q0 = ep.block_tab(kPair02, kPurReluTriple, 0, r2_s, k.rk);
    Lane a0, b0, c0;
    if (sizeof(Lane) == 4) {
      a0 = (Lane)q0.x; b0 = (Lane)q0.y; c0 = (Lane)q0.z;
    } else {
      const U32x4 q2 = ep.block_tab(kPair02, kPurReluTriple, 1, r2_s, k.rk);
      a0 = block_elem<Lane>(q0, 0); b0 = block_elem<Lane>(q0, 1); c0 = block_elem<Lane>(q2, 0);
    }
    a0 &= mask; b0 &= mask; c0 &= mask;
    xd = (Lane)(d * (e + b0) + e * a0 + c0) & mask;
  } else {
    const U32x4 q1 = ep.block_tab(kPair12, kPurReluTriple, 0, r2_s, k.rk);
    const Lane a1 = block_elem<Lane>(q1, 0) & mask, b1 = block_elem<Lane>(q1, 1) & mask;
    xd = (Lane)(d * b1 + e * a1 + lane_at<Lane>(a.pre_c1, i)) & mask;
  }
  lane_put<Lane>(a.out[party], i, t ? (Lane)(s - xd) & mask : xd);
}

// dynamic shared memory of the P2 kernel: two messages of kWarps groups
inline size_t helper_smem_bytes(uint32_t lx) {
  return 2ull * kWarps * (lx + 1) * (lx + 1) * sizeof(uint32_t);
}

template <typename Lane, bool RELU>
cudaError_t launch_stage_t(const PartyArgs& a, int stage, cudaStream_t s) {
  const uint64_t blocks = (a.n + kPB - 1) / kPB;
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  const unsigned parties = a.party0 == kBothParties ? 2u : 1u;
  PartyArgs b = a;
  if (a.party0 == kBothParties) b.party0 = 0;
  if (stage == 1) {
    parties_local_kernel<Lane, RELU><<<dim3((unsigned)blocks, parties), kPB, 0, s>>>(b);
  } else if (stage == 2) {
    // above 48 KB (lx >= 27) the kernel needs the opt-in, which is per device:
    // set it on the current device at each such launch
    const size_t smem = helper_smem_bytes(a.k.lx);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(
          helper_kernel<Lane, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    helper_kernel<Lane, RELU><<<(unsigned)blocks, kPB, smem, s>>>(b);
  } else {
    parties_finish_kernel<Lane, RELU><<<dim3((unsigned)blocks, parties), kPB, 0, s>>>(b);
  }
  return cudaGetLastError();
}

cudaError_t launch_stage(const PartyArgs& a, bool relu, int stage, cudaStream_t s) {
  if (a.k.ring_bits > 32)
    return relu ? launch_stage_t<uint64_t, true>(a, stage, s)
                : launch_stage_t<uint64_t, false>(a, stage, s);
  return relu ? launch_stage_t<uint32_t, true>(a, stage, s)
              : launch_stage_t<uint32_t, false>(a, stage, s);
}

}  // namespace

uint64_t party_msg_words(uint32_t lx, uint64_t n) {
  const uint64_t groups = (n + kPB - 1) / kPB * kWarps;   // padded to whole CTAs
  return (uint64_t)(lx + 1) * groups * (lx + 1);
}

cudaError_t launch_parties(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                           uint64_t n, void* o0, void* o1, uint32_t* w0, uint32_t* w1,
                           void* open0, void* open1, void* reply, void* pre_c1, int* status,
                           bool drop_copies, cudaStream_t s) {
  PartyArgs a{};
  a.k = k;
  a.sh[0] = sh0;
  a.sh[1] = sh1;
  a.out[0] = o0;
  a.out[1] = o1;
  a.w[0] = w0;
  a.w[1] = w1;
  a.open[0] = open0;
  a.open[1] = open1;
  a.reply = reply;
  a.pre_c1 = pre_c1;
  a.n = n;
  a.status = status;
  a.drop_copies = drop_copies ? 1u : 0u;
  a.wait_ns = drop_copies ? kTestWaitNs : kWaitNs;
  a.party0 = kBothParties;
  for (int stage = 1; stage <= 3; ++stage) {
    const cudaError_t e = launch_stage(a, relu, stage, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_party_stage(const ReluConsts& k, bool relu, int stage, int party,
                               const PartyIo& io, uint64_t n, int* status, bool drop_copies,
                               cudaStream_t s) {
  PartyArgs a{};
  a.k = k;
  a.sh[0] = io.sh[0];
  a.sh[1] = io.sh[1];
  a.out[0] = io.out[0];
  a.out[1] = io.out[1];
  a.w[0] = io.w[0];
  a.w[1] = io.w[1];
  a.open[0] = io.open[0];
  a.open[1] = io.open[1];
  a.reply = io.reply;
  a.pre_c1 = io.pre_c1;
  a.n = n;
  a.status = status;
  a.drop_copies = drop_copies ? 1u : 0u;
  a.wait_ns = drop_copies ? kTestWaitNs : kWaitNs;
  a.party0 = (uint32_t)party;
  return launch_stage(a, relu, stage, s);
}

}  // namespace bc
