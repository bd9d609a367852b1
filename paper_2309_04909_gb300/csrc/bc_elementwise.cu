// Elementwise kernels of the hot path: dealer sharing and reconstruction
// (Sec. 2.2), the non-interactive truncations (Alg. smltrc, Alg. newtrc2),
// the modulo switch (Alg. modswitch), Beaver multiplication, and the
// truncation-failure counter used for evaluation.
//
// These are HBM-bound: each thread moves 16 bytes per array per iteration
// (one 128-bit load of 2 x uint64 or 4 x uint32 lanes) when every array is
// 16-byte aligned; grid = SMs x resident CTAs, grid-stride.
#include <type_traits>

#include "bc_internal.h"

namespace bc {
namespace {

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
  T v[V];
};

inline unsigned grid_for(uint64_t work_items, int num_sms, int per_sm) {
  const uint64_t need = (work_items + kBlock - 1) / kBlock;
  const uint64_t full = (uint64_t)num_sms * (uint64_t)per_sm;
  return (unsigned)(need < full ? need : full);
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Generic two-in/two-out elementwise map with V lanes per thread-iteration.
// Op::apply(a, b, index, &oa, &ob).
template <typename In, typename Out, int V, typename Op>
__global__ void __launch_bounds__(kBlock)
    map2_kernel(Op op, const In* __restrict__ a, const In* __restrict__ b, uint64_t n,
                Out* __restrict__ oa, Out* __restrict__ ob) {
  const uint64_t nv = n / V;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t g = (uint64_t)blockIdx.x * kBlock + threadIdx.x; g < nv; g += stride) {
    const Vec<In, V> va = reinterpret_cast<const Vec<In, V>*>(a)[g];
    const Vec<In, V> vb = reinterpret_cast<const Vec<In, V>*>(b)[g];
    Vec<Out, V> ra, rb;
#pragma unroll
    for (int q = 0; q < V; ++q) op.apply(va.v[q], vb.v[q], g * V + q, ra.v[q], rb.v[q]);
    reinterpret_cast<Vec<Out, V>*>(oa)[g] = ra;
    if (ob) reinterpret_cast<Vec<Out, V>*>(ob)[g] = rb;
  }
  // ragged tail (< V elements), taken by the first threads of the grid
  const uint64_t tail = nv * V + (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (tail < n) {
    Out ra, rb;
    op.apply(a[tail], b[tail], tail, ra, rb);
    oa[tail] = ra;
    if (ob) ob[tail] = rb;
  }
}

template <typename In, typename Out, typename Op>
cudaError_t launch_map2(const Op& op, const void* a, const void* b, uint64_t n, void* oa,
                        void* ob, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  constexpr int V = 16 / sizeof(In);
  const bool vec = aligned16(a) && aligned16(b) && aligned16(oa) && (!ob || aligned16(ob)) &&
                   (sizeof(Out) * V) % 8 == 0;
  if (vec) {
    auto kern = map2_kernel<In, Out, V, Op>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
    unsigned g = grid_for(n / V > 0 ? n / V : 1, num_sms, per_sm < 1 ? 1 : per_sm);
    kern<<<g, kBlock, 0, s>>>(op, static_cast<const In*>(a), static_cast<const In*>(b), n,
                              static_cast<Out*>(oa), static_cast<Out*>(ob));
  } else {
    auto kern = map2_kernel<In, Out, 1, Op>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
    unsigned g = grid_for(n, num_sms, per_sm < 1 ? 1 : per_sm);
    kern<<<g, kBlock, 0, s>>>(op, static_cast<const In*>(a), static_cast<const In*>(b), n,
                              static_cast<Out*>(oa), static_cast<Out*>(ob));
  }
  return cudaGetLastError();
}

// ---- reconstruction: x = [x]_0 + [x]_1 mod 2^l ------------------------------
template <typename Lane>
struct ReconstructOp {
  Lane mask;
  __device__ __forceinline__ void apply(Lane a, Lane b, uint64_t, Lane& o, Lane& u) const {
    o = (Lane)(a + b) & mask;
    u = 0;
  }
};

// ---- Alg. smltrc: P0 cut([x]_0,k); P1 2^l - cut(2^l - [x]_1, k) ------------
template <typename Lane>
struct TruncProbOp {
  Lane mask;
  uint32_t k;
  __device__ __forceinline__ void apply(Lane a, Lane b, uint64_t, Lane& o0, Lane& o1) const {
    o0 = a >> k;
    o1 = ring_neg<Lane>((Lane)(ring_neg<Lane>(b, mask) >> k), mask);
  }
};

// ---- Alg. newtrc2: keep bits k1 .. l-k2-1, outputs mod 2^(l-k1-k2) --------
template <typename In, typename Out>
struct TruncDetOp {
  In mask;          // 2^l - 1
  Out omask;        // 2^(l-k1-k2) - 1
  uint32_t k1;
  __device__ __forceinline__ void apply(In a, In b, uint64_t, Out& o0, Out& o1) const {
    o0 = (Out)(a >> k1) & omask;
    const Out c = (Out)(ring_neg<In>(b, mask) >> k1);
    o1 = (Out)(Out(0) - c) & omask;
  }
};

// ---- Alg. modswitch: Z_{2^lp} -> Z_p (p > 2^lp) ------------------------------
struct ModSwitchOp {
  uint32_t lmask;   // 2^lp - 1
  uint32_t two_lp;  // 2^lp (< p, so also 2^lp mod p)
  uint32_t p;
  __device__ __forceinline__ void apply(uint32_t a, uint32_t b, uint64_t, uint32_t& o0,
                                        uint32_t& o1) const {
    a &= lmask;
    b &= lmask;
    o0 = a ? a : two_lp;            // a < 2^lp < p
    o1 = b + (p - two_lp);          // p + b - 2^lp in [p - 2^lp, p)
  }
};

// ---- dealer sharing -------------------------------------------------------
template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    share_kernel(const RoundKeys rk, const int64_t* __restrict__ x, uint64_t n, uint32_t tid,
                 uint64_t base, Lane mask, Lane* __restrict__ s0, Lane* __restrict__ s1) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
    const U32x4 b = draw_block(kPairDealer, kPurShare, tid, base + i, 0, rk);
    const Lane R = block_elem<Lane>(b, 0) & mask;
    s0[i] = (Lane)((Lane)x[i] + R) & mask;
    s1[i] = ring_neg<Lane>(R, mask);
  }
}

// ---- Beaver multiplication -------------------------------------------------
template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    mul_beaver_kernel(const RoundKeys rk, Lane mask, uint32_t tid, uint64_t base,
                      const Lane* __restrict__ x0,
                      const Lane* __restrict__ x1, const Lane* __restrict__ y0,
                      const Lane* __restrict__ y1, uint64_t n, Lane* __restrict__ o0,
                      Lane* __restrict__ o1) {
  __shared__ uint64_t r2_s[2];   // round2_product(tid, b) for the triple's blocks b = 0, 1
  if (threadIdx.x < 2) r2_s[threadIdx.x] = round2_product(tid, threadIdx.x, rk);
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
    Lane p0, p1;
    beaver_mul<Lane>(ElemPhilox(base + i, tid), rk, mask, x0[i], x1[i], y0[i], y1[i], p0, p1,
                     r2_s);
    o0[i] = p0;
    o1[i] = p1;
  }
}

// ---- Alg. aby3trc: open alpha = x + r, P0: alpha / 2^k - [r']_0, P1: -[r']_1 ---
// floor(signed(a) / 2^k) in Z_{2^l}: sign-extend bit l-1, arithmetic shift.
template <typename Lane>
__device__ __forceinline__ Lane sdiv_pow2(Lane a, Lane mask, uint32_t ell, uint32_t k) {
  using S = typename std::conditional<sizeof(Lane) == 8, int64_t, int32_t>::type;
  const Lane sign = (Lane)1 << (ell - 1);
  const S v = (S)((a ^ sign) - sign);   // two's-complement value of the l-bit a
  return (Lane)(v >> k) & mask;
}

template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    aby3_trunc_kernel(const RoundKeys rk, Lane mask, uint32_t ell, uint32_t k, uint32_t tid,
                      uint64_t base, Lane fixed_r, const Lane* __restrict__ s0,
                      const Lane* __restrict__ s1, uint64_t n, Lane* __restrict__ o0,
                      Lane* __restrict__ o1) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
    const uint64_t elem = base + i;
    const U32x4 q02 = draw_block(kPair02, kPurAby3, tid, elem, 0, rk);   // P0 and P2
    const U32x4 q12 = draw_block(kPair12, kPurAby3, tid, elem, 0, rk);   // P1 and P2
    const Lane r0 = block_elem<Lane>(q02, 0) & mask;
    const Lane rp0 = block_elem<Lane>(q02, 1) & mask;
    Lane r1 = block_elem<Lane>(q12, 0) & mask;
    if (fixed_r) r1 = (Lane)(fixed_r - r0) & mask;
    // P2: r' = r / 2^k, [r']_1 = r' - [r']_0 -> P1
    const Lane rp1 = (Lane)(sdiv_pow2<Lane>((Lane)(r0 + r1) & mask, mask, ell, k) - rp0) & mask;
    // P0 and P1 open alpha = ([x]_0 + [r]_0) + ([x]_1 + [r]_1)
    const Lane alpha = (Lane)((s0[i] + r0) + (s1[i] + r1)) & mask;
    o0[i] = (Lane)(sdiv_pow2<Lane>(alpha, mask, ell, k) - rp0) & mask;
    o1[i] = ring_neg<Lane>(rp1, mask);
  }
}

// ---- Alg. linear: Alg. smltrc on both inputs, then the Beaver product --------
template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    trunc_then_mul_kernel(const RoundKeys rk, Lane mask, uint32_t kx, uint32_t ky, uint32_t tid,
                          uint64_t base, const Lane* __restrict__ x0, const Lane* __restrict__ x1,
                          const Lane* __restrict__ y0, const Lane* __restrict__ y1, uint64_t n,
                          Lane* __restrict__ o0, Lane* __restrict__ o1) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
    const Lane tx0 = x0[i] >> kx;
    const Lane tx1 = ring_neg<Lane>((Lane)(ring_neg<Lane>(x1[i], mask) >> kx), mask);
    const Lane ty0 = y0[i] >> ky;
    const Lane ty1 = ring_neg<Lane>((Lane)(ring_neg<Lane>(y1[i], mask) >> ky), mask);
    const uint64_t elem = base + i;
    const U32x4 q0 = draw_block(kPair02, kPurMulTriple, tid, elem, 0, rk);
    const U32x4 q1 = draw_block(kPair12, kPurMulTriple, tid, elem, 0, rk);
    Lane a0, b0, c0;
    if (sizeof(Lane) == 4) {
      a0 = (Lane)q0.x; b0 = (Lane)q0.y; c0 = (Lane)q0.z;
    } else {
      const U32x4 q2 = draw_block(kPair02, kPurMulTriple, tid, elem, 1, rk);
      a0 = block_elem<Lane>(q0, 0); b0 = block_elem<Lane>(q0, 1); c0 = block_elem<Lane>(q2, 0);
    }
    const Lane a1 = block_elem<Lane>(q1, 0) & mask, b1 = block_elem<Lane>(q1, 1) & mask;
    a0 &= mask; b0 &= mask; c0 &= mask;
    const Lane c1 = (Lane)((a0 + a1) * (b0 + b1) - c0) & mask;
    const Lane d = (Lane)((tx0 - a0) + (tx1 - a1)) & mask;
    const Lane e = (Lane)((ty0 - b0) + (ty1 - b1)) & mask;
    o0[i] = (Lane)(d * e + d * b0 + e * a0 + c0) & mask;
    o1[i] = (Lane)(d * b1 + e * a1 + c1) & mask;
  }
}

// ---- truncation failures vs the plaintext ---------------------------------
template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    count_failures_kernel(Lane omask, uint32_t k, const int64_t* __restrict__ x,
                          const Lane* __restrict__ o0, const Lane* __restrict__ o1, uint64_t n,
                          unsigned long long* __restrict__ count) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  unsigned long long local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
    const Lane rec = (Lane)(o0[i] + o1[i]) & omask;
    const Lane want = (Lane)(x[i] >> k) & omask;   // floor(x / 2^k) mod 2^out
    const Lane d = (Lane)(rec - want) & omask;
    local += (d != 0 && d != 1 && d != omask) ? 1ull : 0ull;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

template <typename Lane>
Lane lane_mask(int bits) {
  return bits >= (int)(8 * sizeof(Lane)) ? (Lane)~(Lane)0 : (Lane)(((Lane)1 << bits) - 1);
}

template <typename K>
unsigned simple_grid(K kern, uint64_t n, int num_sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
  return grid_for(n, num_sms, per_sm < 1 ? 1 : per_sm);
}

}  // namespace

cudaError_t launch_reconstruct(int ring_bits, const void* sh0, const void* sh1, uint64_t n,
                               void* out, int num_sms, cudaStream_t s) {
  if (ring_bits > 32)
    return launch_map2<uint64_t, uint64_t>(ReconstructOp<uint64_t>{lane_mask<uint64_t>(ring_bits)},
                                           sh0, sh1, n, out, nullptr, num_sms, s);
  return launch_map2<uint32_t, uint32_t>(ReconstructOp<uint32_t>{lane_mask<uint32_t>(ring_bits)},
                                         sh0, sh1, n, out, nullptr, num_sms, s);
}

cudaError_t launch_trunc_prob(int ring_bits, int k, const void* sh0, const void* sh1, uint64_t n,
                              void* o0, void* o1, int num_sms, cudaStream_t s) {
  if (ring_bits > 32)
    return launch_map2<uint64_t, uint64_t>(
        TruncProbOp<uint64_t>{lane_mask<uint64_t>(ring_bits), (uint32_t)k}, sh0, sh1, n, o0, o1,
        num_sms, s);
  return launch_map2<uint32_t, uint32_t>(
      TruncProbOp<uint32_t>{lane_mask<uint32_t>(ring_bits), (uint32_t)k}, sh0, sh1, n, o0, o1,
      num_sms, s);
}

cudaError_t launch_trunc_det(int ring_bits, int k1, int k2, const void* sh0, const void* sh1,
                             uint64_t n, void* o0, void* o1, int num_sms, cudaStream_t s) {
  const int ob = ring_bits - k1 - k2;
  if (ring_bits > 32) {
    if (ob > 32)
      return launch_map2<uint64_t, uint64_t>(
          TruncDetOp<uint64_t, uint64_t>{lane_mask<uint64_t>(ring_bits), lane_mask<uint64_t>(ob),
                                         (uint32_t)k1},
          sh0, sh1, n, o0, o1, num_sms, s);
    return launch_map2<uint64_t, uint32_t>(
        TruncDetOp<uint64_t, uint32_t>{lane_mask<uint64_t>(ring_bits), lane_mask<uint32_t>(ob),
                                       (uint32_t)k1},
        sh0, sh1, n, o0, o1, num_sms, s);
  }
  return launch_map2<uint32_t, uint32_t>(
      TruncDetOp<uint32_t, uint32_t>{lane_mask<uint32_t>(ring_bits), lane_mask<uint32_t>(ob),
                                     (uint32_t)k1},
      sh0, sh1, n, o0, o1, num_sms, s);
}

cudaError_t launch_mod_switch(int lp, uint32_t p, const void* sh0, const void* sh1, uint64_t n,
                              uint32_t* o0, uint32_t* o1, int num_sms, cudaStream_t s) {
  const ModSwitchOp op{lane_mask<uint32_t>(lp), 1u << lp, p};
  return launch_map2<uint32_t, uint32_t>(op, sh0, sh1, n, o0, o1, num_sms, s);
}

cudaError_t launch_share(int ring_bits, const RoundKeys& rk, const int64_t* x, uint64_t n,
                         uint32_t tensor_id, uint64_t elem_base, void* sh0, void* sh1, int num_sms,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (ring_bits > 32) {
    auto kern = share_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, x, n, tensor_id, elem_base, lane_mask<uint64_t>(ring_bits), static_cast<uint64_t*>(sh0),
        static_cast<uint64_t*>(sh1));
  } else {
    auto kern = share_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, x, n, tensor_id, elem_base, lane_mask<uint32_t>(ring_bits), static_cast<uint32_t*>(sh0),
        static_cast<uint32_t*>(sh1));
  }
  return cudaGetLastError();
}

// Lanes of a share array with bits at or above l set (checked mode).
template <typename Lane>
__global__ void __launch_bounds__(kBlock)
    noncanonical_kernel(const Lane* __restrict__ a, uint64_t n, uint32_t ell,
                        unsigned long long* __restrict__ count) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  unsigned int bad = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride)
    bad += (a[i] >> ell) != 0 ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, (unsigned long long)bad);
}

cudaError_t launch_count_noncanonical(int ring_bits, const void* a, uint64_t n,
                                      unsigned long long* count, int num_sms, cudaStream_t s) {
  if (n == 0 || ring_bits == 32 || ring_bits == 64) return cudaSuccess;   // every lane fits
  if (ring_bits > 32) {
    auto kern = noncanonical_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(static_cast<const uint64_t*>(a), n,
                                                          (uint32_t)ring_bits, count);
  } else {
    auto kern = noncanonical_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(static_cast<const uint32_t*>(a), n,
                                                          (uint32_t)ring_bits, count);
  }
  return cudaGetLastError();
}

cudaError_t launch_mul_beaver(int ring_bits, const RoundKeys& rk, const void* x0, const void* x1,
                              const void* y0, const void* y1, uint64_t n, uint32_t tensor_id,
                              uint64_t elem_base, void* o0, void* o1, int num_sms,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (ring_bits > 32) {
    auto kern = mul_beaver_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint64_t>(ring_bits), tensor_id, elem_base, static_cast<const uint64_t*>(x0),
        static_cast<const uint64_t*>(x1), static_cast<const uint64_t*>(y0),
        static_cast<const uint64_t*>(y1), n, static_cast<uint64_t*>(o0),
        static_cast<uint64_t*>(o1));
  } else {
    auto kern = mul_beaver_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint32_t>(ring_bits), tensor_id, elem_base, static_cast<const uint32_t*>(x0),
        static_cast<const uint32_t*>(x1), static_cast<const uint32_t*>(y0),
        static_cast<const uint32_t*>(y1), n, static_cast<uint32_t*>(o0),
        static_cast<uint32_t*>(o1));
  }
  return cudaGetLastError();
}

cudaError_t launch_trunc_aby3(int ring_bits, const RoundKeys& rk, int k, const void* sh0,
                              const void* sh1, uint64_t n, uint32_t tensor_id, uint64_t fixed_r,
                              void* o0, void* o1, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (ring_bits > 32) {
    auto kern = aby3_trunc_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint64_t>(ring_bits), (uint32_t)ring_bits, (uint32_t)k, tensor_id, 0,
        (uint64_t)fixed_r, static_cast<const uint64_t*>(sh0), static_cast<const uint64_t*>(sh1), n,
        static_cast<uint64_t*>(o0), static_cast<uint64_t*>(o1));
  } else {
    auto kern = aby3_trunc_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint32_t>(ring_bits), (uint32_t)ring_bits, (uint32_t)k, tensor_id, 0,
        (uint32_t)fixed_r, static_cast<const uint32_t*>(sh0), static_cast<const uint32_t*>(sh1), n,
        static_cast<uint32_t*>(o0), static_cast<uint32_t*>(o1));
  }
  return cudaGetLastError();
}

cudaError_t launch_trunc_then_mul(int ring_bits, const RoundKeys& rk, int kx, int ky,
                                  const void* x0, const void* x1, const void* y0, const void* y1,
                                  uint64_t n, uint32_t tensor_id, void* o0, void* o1, int num_sms,
                                  cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (ring_bits > 32) {
    auto kern = trunc_then_mul_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint64_t>(ring_bits), (uint32_t)kx, (uint32_t)ky, tensor_id, 0,
        static_cast<const uint64_t*>(x0), static_cast<const uint64_t*>(x1),
        static_cast<const uint64_t*>(y0), static_cast<const uint64_t*>(y1), n,
        static_cast<uint64_t*>(o0), static_cast<uint64_t*>(o1));
  } else {
    auto kern = trunc_then_mul_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        rk, lane_mask<uint32_t>(ring_bits), (uint32_t)kx, (uint32_t)ky, tensor_id, 0,
        static_cast<const uint32_t*>(x0), static_cast<const uint32_t*>(x1),
        static_cast<const uint32_t*>(y0), static_cast<const uint32_t*>(y1), n,
        static_cast<uint32_t*>(o0), static_cast<uint32_t*>(o1));
  }
  return cudaGetLastError();
}

cudaError_t launch_count_failures(int out_bits, int k, const int64_t* x, const void* o0,
                                  const void* o1, uint64_t n, unsigned long long* count,
                                  int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (out_bits > 32) {
    auto kern = count_failures_kernel<uint64_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        lane_mask<uint64_t>(out_bits), (uint32_t)k, x, static_cast<const uint64_t*>(o0),
        static_cast<const uint64_t*>(o1), n, count);
  } else {
    auto kern = count_failures_kernel<uint32_t>;
    kern<<<simple_grid(kern, n, num_sms), kBlock, 0, s>>>(
        lane_mask<uint32_t>(out_bits), (uint32_t)k, x, static_cast<const uint32_t*>(o0),
        static_cast<const uint32_t*>(o1), n, count);
  }
  return cudaGetLastError();
}

}  // namespace bc
