// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bicoptor.h"
#include "bc_device.cuh"

namespace bc {

constexpr int kBlock = 256;     // threads per CTA of every kernel
constexpr int kMaxSlots = 32;   // lx + 1 <= 32

// The Philox counter carries 48 bits of the element index (word 0 and the low
// 16 bits of word 3), so the elements of one tensor id are numbered below 2^48.
constexpr uint64_t kMaxElemIndex = 1ull << 48;
inline bool elem_range_ok(uint64_t first, uint64_t n) {
  return first <= kMaxElemIndex && n <= kMaxElemIndex - first;
}

// Per-call constants of Alg. drelu / Alg. relu, passed by value.
struct ReluConsts {
  RoundKeys rk;
  ModP mp;
  uint64_t ring_mask;   // 2^l - 1 (as the lane type)
  uint32_t ring_bits;
  uint32_t lx;          // key bits
  uint32_t c;           // key offset
  uint32_t mx;          // 2^lx - 1
  uint32_t two_lx;      // 2^lx (= 2^lx mod p, since p > 2^lx)
  uint32_t p_minus_2lx; // p - 2^lx
  uint32_t tensor_id;
  uint64_t elem_base;   // element index of the launch's first element
  // Always 0 and 2^32 - p: operands the compiler cannot fold, which keep the
  // slot loop's sums in three-input form (see BC_ALU_ADDS in bc_element.cuh).
  uint32_t zero1, zero2, neg_p;
};

struct AuditPtrs {
  uint32_t* w0;
  uint32_t* w1;
  void* reply;
  void* open0;
  void* open1;
  void* pre_c1;
  uint8_t* t;
  uint8_t* dprime;
  bool any() const { return w0 || w1 || reply || open0 || open1 || pre_c1 || t || dprime; }
};

// One tensor of a batched launch, resident in device memory.  The protocol
// constants are shared by every tensor of a parameter group and travel as a
// kernel parameter (ReluConsts), not per tensor.
struct BatchTensor {
  const void* sh0;
  const void* sh1;
  void* o0;
  void* o1;
  uint64_t n;
  uint32_t tensor_id;
  int op;              // BC_OP_RELU / BC_OP_DRELU
  uint64_t elem_offset;  // Philox element index of element 0
  uint32_t first_tile;   // index of the tensor's first tile in the tile table
};

struct BatchTile {
  uint32_t tensor;     // index into the tensor table
  uint32_t count;      // elements in this tile
  uint64_t start;      // first element of the tile within its tensor
};

// A parameter group: tensors with the same (l, lx, c, p) own the tiles
// [begin, end) of the table and run as one persistent kernel.
constexpr int kMaxBatchGroups = 32;
struct BatchGroup {
  ReluConsts k;        // tensor_id / elem_base unused
  uint32_t begin, end;
};

// ---- host helpers shared by the context path (bc_api.cu) and the
// allocation-free path (bc_noalloc.cu) ----------------------------------------

inline bool is_prime_u32(uint64_t q) {
  if (q < 2) return false;
  if (q % 2 == 0) return q == 2;
  for (uint64_t d = 3; d * d <= q; d += 2)
    if (q % d == 0) return false;
  return true;
}

inline uint64_t ring_mask(int bits) {
  return bits >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1);
}

// Philox-4x32-10 round keys of a 64-bit seed: key (lo32, hi32) plus the
// Weyl increments of each round.
inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return rk;
}

// Montgomery constants of p (R = 2^32).
inline ModP make_modp(uint32_t p) {
  ModP m;
  m.p = p;
  uint32_t inv = p;                      // Newton: inv = p^{-1} mod 2^32
  for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
  m.pinv = 0u - inv;
  const uint64_t r1 = ((uint64_t)1 << 32) % p;
  m.r2 = (uint32_t)((r1 * r1) % p);
  m.pm1 = p - 1;
  return m;
}

// The last (lx, p) pairs whose p passed the primality test, so that a call
// does not repeat the trial division (up to 2^15.5 divisions at lx = 31).
struct PrimeCache {
  uint32_t p[4] = {0, 0, 0, 0};
  int lx[4] = {0, 0, 0, 0};
  int next = 0;
  bool prime(uint32_t q, int l) {
    for (int i = 0; i < 4; ++i)
      if (p[i] == q && lx[i] == l) return true;
    if (!is_prime_u32(q)) return false;
    p[next] = q;
    lx[next] = l;
    next = (next + 1) & 3;
    return true;
  }
};

// Checks of Alg. drelu's parameters (c + 2 lx <= l, p a prime in
// (2^lx, 2^(lx+1)); p = 0 takes the smallest one) and the kernel constants of
// a tensor.  BC_OK or BC_EINVAL.
inline int make_relu_consts(const bc_drelu_params* prm, const RoundKeys& rk, uint32_t tensor_id,
                            PrimeCache& primes, ReluConsts* k) {
  if (!prm) return BC_EINVAL;
  const int ell = prm->ring_bits, lx = prm->lx, c = prm->key_off;
  if (ell < 2 || ell > 64 || lx < 1 || lx > 31 || c < 0 || c + 2 * lx > ell) return BC_EINVAL;
  const uint32_t p = prm->p ? prm->p : bc_prime_above(lx);
  const uint64_t lo = (uint64_t)1 << lx, hi = (uint64_t)1 << (lx + 1);
  if ((uint64_t)p <= lo || (uint64_t)p >= hi || !primes.prime(p, lx)) return BC_EINVAL;
  k->rk = rk;
  k->mp = make_modp(p);
  k->ring_mask = ring_mask(ell);
  k->ring_bits = (uint32_t)ell;
  k->lx = (uint32_t)lx;
  k->c = (uint32_t)c;
  k->mx = (uint32_t)(lo - 1);
  k->two_lx = (uint32_t)lo;
  k->p_minus_2lx = p - (uint32_t)lo;
  k->tensor_id = tensor_id;
  k->elem_base = 0;
  k->zero1 = k->zero2 = 0;
  k->neg_p = 0u - p;
  return BC_OK;
}

// Host-side launchers (return cudaError_t of the launch).
cudaError_t launch_relu(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                        uint64_t n, void* o0, void* o1, const AuditPtrs& aud, int num_sms,
                        cudaStream_t s);
// Launch shape of a batched run.  ctas_per_sm >= 0: persistent schedule
// (0 = occupancy).  ctas_per_sm < 0: grid schedule, one CTA per tile of at
// most kBlock * elems_per_thread elements (1, 2 or 4).  slot_unroll: unroll of
// the key-bit loop (1, 2 or 3; 0 = default).
struct BatchLaunch {
  int ctas_per_sm;
  int elems_per_thread;
  int slot_unroll;
};
// Writes the tile table of a planned batch on the device: tiles of `tile`
// elements, tensor by tensor in table order, tensor t's tiles starting at
// tensors[t].first_tile (non-decreasing, tensors[0].first_tile = 0), ntiles in
// all.  The host plans O(tensors) work; the table itself is built here.
cudaError_t launch_expand_tiles(const BatchTensor* tensors, uint32_t count, uint32_t ntiles,
                                uint32_t tile, BatchTile* tiles, cudaStream_t s);
// Launches one kernel per non-empty group; for the persistent schedule
// `counters` holds one zeroed work counter per group.
cudaError_t launch_relu_batch(const BatchTensor* tensors, const BatchTile* tiles,
                              const BatchGroup* groups, int ngroups, unsigned int* counters,
                              int* status, int num_sms, const BatchLaunch& launch,
                              cudaStream_t s);

// The fused step of a linear layer followed by a ReLU: Beaver product of
// [x][y], Alg. smltrc and Alg. newtrc2 of the product by `trunc` bits, and
// Alg. relu of the probabilistically truncated product.
struct LinearConsts {
  ReluConsts k;         // ReLU constants; k.tensor_id is the ReLU's id, k.elem_base the
                        // element index of the launch's first element (product and ReLU)
  uint32_t mul_tid;     // tensor id of the product's triple
  uint32_t trunc;       // truncation bits
  uint64_t det_mask;    // 2^(l - trunc) - 1
  uint32_t det_wide;    // l - trunc > 32: 64-bit lanes for the deterministic truncation
};
struct LinearIo {
  const void *x0, *x1, *y0, *y1;   // input shares
  void *prod0, *prod1;             // product shares (optional)
  void *trc0, *trc1;               // probabilistic truncation (optional)
  void *det0, *det1;               // deterministic truncation (optional)
  void *relu0, *relu1;             // ReLU shares
};
cudaError_t launch_linear_relu(const LinearConsts& c, const LinearIo& io, uint64_t n,
                               cudaStream_t s);

// Alg. drelu2 / RSS ReLU on replicated components x[0..2] -> y[0..2].
cudaError_t launch_rss(const ReluConsts& k, bool relu, const void* const* x, uint64_t n,
                       void* const* y, cudaStream_t s);

// Party-separated DReLU/ReLU (three launches, messages in device buffers).
uint64_t party_msg_words(uint32_t lx, uint64_t n);
// `status` is set to BC_ETIMEOUT if P2's kernel gives up waiting for its
// messages; drop_copies (testing only) makes it issue no copies so that it does.
cudaError_t launch_parties(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                           uint64_t n, void* o0, void* o1, uint32_t* w0, uint32_t* w1,
                           void* open0, void* open1, void* reply, void* pre_c1, int* status,
                           bool drop_copies, cudaStream_t s);

// One stage of a party-separated call run by one party (P0 or P1 for stages
// 1 and 3, P2 for stage 2), for callers that keep the parties in separate
// processes and move the messages between the stages themselves.  Only the
// buffers of that party's stage are read or written.
struct PartyIo {
  const void* sh[2];
  void* out[2];
  uint32_t* w[2];
  void* open[2];
  void* reply;
  void* pre_c1;
};
cudaError_t launch_party_stage(const ReluConsts& k, bool relu, int stage, int party,
                               const PartyIo& io, uint64_t n, int* status, bool drop_copies,
                               cudaStream_t s);

// The Bicoptor 1.0-style DReLU / ReLU (bc_b1.cu); w0, w1 (optional) receive
// the messages, n * (lx + 1) lanes each, slot-major per element.
cudaError_t launch_b1(const ReluConsts& k, bool relu, const void* sh0, const void* sh1,
                      uint64_t n, void* o0, void* o1, void* w0, void* w1, cudaStream_t s);

cudaError_t launch_share(int ring_bits, const RoundKeys& rk, const int64_t* x, uint64_t n,
                         uint32_t tensor_id, uint64_t elem_base, void* sh0, void* sh1, int num_sms,
                         cudaStream_t s);
cudaError_t launch_reconstruct(int ring_bits, const void* sh0, const void* sh1, uint64_t n,
                               void* out, int num_sms, cudaStream_t s);
cudaError_t launch_trunc_prob(int ring_bits, int k, const void* sh0, const void* sh1, uint64_t n,
                              void* o0, void* o1, int num_sms, cudaStream_t s);
cudaError_t launch_trunc_det(int ring_bits, int k1, int k2, const void* sh0, const void* sh1,
                             uint64_t n, void* o0, void* o1, int num_sms, cudaStream_t s);
cudaError_t launch_mod_switch(int lp, uint32_t p, const void* sh0, const void* sh1, uint64_t n,
                              uint32_t* o0, uint32_t* o1, int num_sms, cudaStream_t s);
cudaError_t launch_mul_beaver(int ring_bits, const RoundKeys& rk, const void* x0, const void* x1,
                              const void* y0, const void* y1, uint64_t n, uint32_t tensor_id,
                              uint64_t elem_base, void* o0, void* o1, int num_sms,
                              cudaStream_t s);
cudaError_t launch_trunc_aby3(int ring_bits, const RoundKeys& rk, int k, const void* sh0,
                              const void* sh1, uint64_t n, uint32_t tensor_id, uint64_t fixed_r,
                              void* o0, void* o1, int num_sms, cudaStream_t s);
cudaError_t launch_trunc_then_mul(int ring_bits, const RoundKeys& rk, int kx, int ky,
                                  const void* x0, const void* x1, const void* y0, const void* y1,
                                  uint64_t n, uint32_t tensor_id, void* o0, void* o1, int num_sms,
                                  cudaStream_t s);
cudaError_t launch_count_noncanonical(int ring_bits, const void* a, uint64_t n,
                                      unsigned long long* count, int num_sms, cudaStream_t s);
cudaError_t launch_count_failures(int out_bits, int k, const int64_t* x, const void* o0,
                                  const void* o1, uint64_t n, unsigned long long* count,
                                  int num_sms, cudaStream_t s);

}  // namespace bc
