// Batched DReLU/ReLU over many tensors (the batching of Alg. drelu / Alg.
// relu across a network's layers and requests): one launch per parameter
// group (l, lx, c, p) over that group's range of a tile table.
//
// Two schedules:
//   grid        one CTA per tile of 256 x EPT elements, EPT elements per
//               thread; the hardware CTA scheduler is the queue.
//   persistent  one grid sized to residency whose warps take the next tile
//               from the group's atomic counter (no block barrier, no waits),
//               so uneven tensors balance down to one tile per warp.
// Per-group kernels keep the register allocation of a single variant.  The
// key-bit (message-slot) loop unroll UNROLL and EPT are template parameters
// chosen per plan, so an autotuner can pick them; the key widths of the
// benchmarked workloads (lx = 24 at l = 64, lx = 14 and 9 at l = 32) have
// every variant, other widths take the generic kernel with the default
// unroll.
#include "bc_element.cuh"

// The minimum resident CTAs per SM requested from the register allocator for
// the one-element-per-thread grid kernels of key widths lx >= 14 with the slot
// loop unrolled whole (compile-time; 0 = let it choose).  Left to itself the
// allocator takes 51-52 registers there (4 CTAs of 256 threads); six CTAs
// keep them at 40 registers without spilling, which is faster.  The other
// kernels are left free: shorter loops already fit in 40 registers, the
// partly unrolled loops ran slower under the bound, and the multi-element and
// persistent kernels would spill.
#ifndef BC_BATCH_MIN_CTAS
#define BC_BATCH_MIN_CTAS 6
#endif
// The same for 32-bit lanes (l <= 32): at six CTAs that kernel spills 8 bytes
// at lx = 14; five CTAs give it 48 registers and no spill, 0.15% faster on
// the two-ring ResNet-18 set.
#ifndef BC_BATCH_MIN_CTAS_L32
#define BC_BATCH_MIN_CTAS_L32 5
#endif

namespace bc {
namespace {

template <typename Lane, int LX, bool SHORT, bool RELU, int UNROLL>
__device__ __forceinline__ void run_tile(const ReluConsts& k, const BatchTensor& bt,
                                         uint64_t start, uint32_t count, uint32_t lane,
                                         uint32_t* perm, const uint64_t* r2) {
  const Lane* sh0 = static_cast<const Lane*>(bt.sh0);
  const Lane* sh1 = static_cast<const Lane*>(bt.sh1);
  Lane* o0 = static_cast<Lane*>(bt.o0);
  Lane* o1 = static_cast<Lane*>(bt.o1);
  const AuditPtrs none{};
#pragma unroll 1
  for (uint32_t j = lane; j < count; j += 32) {
    const uint64_t i = start + j;
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, RELU, false, false, UNROLL>(
        k, k.rk, bt.tensor_id, sh0[i], sh1[i], bt.elem_offset + i, perm, r0, r1, none, i, r2);
    o0[i] = r0;
    o1[i] = r1;
  }
}

template <typename Lane, int LX, bool SHORT, int UNROLL>
__global__ void __launch_bounds__(kBlock)
    relu_batch_kernel(const ReluConsts k, const BatchTensor* __restrict__ tensors,
                      const BatchTile* __restrict__ tiles, uint32_t begin, uint32_t end,
                      unsigned int* __restrict__ counter, int* __restrict__ status) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  __shared__ uint64_t r2_s[kBlock / 32][kMaxSlots];   // per warp: its tile's tensor
  uint32_t* perm = perm_s + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t* r2 = r2_s[threadIdx.x >> 5];
  for (;;) {
    uint32_t tile = 0;
    if (lane == 0) tile = begin + atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);   // also: every lane is done with the last tile
    if (tile >= end) break;
    const BatchTile tl = tiles[tile];
    const BatchTensor bt = tensors[tl.tensor];
    if (tl.start + tl.count > bt.n) {   // a malformed table: record, skip
      if (lane == 0) atomicExch(status, BC_ECHECK);
      continue;
    }
    r2[lane] = round2_product(bt.tensor_id, lane, k.rk);   // kMaxSlots == 32 lanes
    __syncwarp();
    if (bt.op == BC_OP_DRELU)
      run_tile<Lane, LX, SHORT, false, UNROLL>(k, bt, tl.start, tl.count, lane, perm, r2);
    else
      run_tile<Lane, LX, SHORT, true, UNROLL>(k, bt, tl.start, tl.count, lane, perm, r2);
  }
}

// Grid schedule: one CTA per tile of at most kBlock * EPT elements; thread t
// takes elements t, t + kBlock, ... of the tile (coalesced at every step).
// EPT = 1 has no loop, so nothing is kept live across elements.
template <typename Lane, int LX, bool SHORT, bool RELU, int UNROLL, int EPT>
__device__ __forceinline__ void grid_tile(const ReluConsts& k, const BatchTensor& bt,
                                          const BatchTile& tl, uint32_t* perm,
                                          const uint64_t* r2) {
  const Lane* sh0 = static_cast<const Lane*>(bt.sh0);
  const Lane* sh1 = static_cast<const Lane*>(bt.sh1);
  Lane* o0 = static_cast<Lane*>(bt.o0);
  Lane* o1 = static_cast<Lane*>(bt.o1);
  const AuditPtrs none{};
  if (EPT == 1) {
    if (threadIdx.x >= tl.count) return;
    const uint64_t i = tl.start + threadIdx.x;
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, RELU, false, false, UNROLL>(
        k, k.rk, bt.tensor_id, sh0[i], sh1[i], bt.elem_offset + i, perm, r0, r1, none, i, r2);
    o0[i] = r0;
    o1[i] = r1;
    return;
  }
#pragma unroll 1
  for (uint32_t j = threadIdx.x; j < tl.count; j += kBlock) {
    const uint64_t i = tl.start + j;
    Lane r0, r1;
    bicoptor_element<Lane, LX, SHORT, RELU, false, false, UNROLL>(
        k, k.rk, bt.tensor_id, sh0[i], sh1[i], bt.elem_offset + i, perm, r0, r1, none, i, r2);
    o0[i] = r0;
    o1[i] = r1;
  }
}

template <typename Lane, int LX, bool SHORT, int UNROLL, int EPT>
__global__ void __launch_bounds__(kBlock, (LX >= 14 && EPT == 1 && UNROLL == 0)
                                              ? (sizeof(Lane) == 8 ? BC_BATCH_MIN_CTAS
                                                                   : BC_BATCH_MIN_CTAS_L32)
                                              : 0)
    relu_batch_grid_kernel(const ReluConsts k, const BatchTensor* __restrict__ tensors,
                           const BatchTile* __restrict__ tiles, uint32_t begin,
                           int* __restrict__ status) {
  __shared__ uint32_t perm_s[(LX ? LX + 1 : kMaxSlots) * kBlock];
  __shared__ uint64_t r2_s[kMaxSlots];   // the tile's tensor: round2_product(tensor_id, b)
  uint32_t* perm = perm_s + threadIdx.x;
  const BatchTile tl = tiles[begin + blockIdx.x];
  const BatchTensor bt = tensors[tl.tensor];
  if (tl.count > (uint32_t)(kBlock * EPT) || tl.start + tl.count > bt.n) {   // malformed: skip
    if (threadIdx.x == 0) atomicExch(status, BC_ECHECK);
    return;
  }
  if (threadIdx.x < kMaxSlots) r2_s[threadIdx.x] = round2_product(bt.tensor_id, threadIdx.x, k.rk);
  __syncthreads();
  if (bt.op == BC_OP_DRELU)
    grid_tile<Lane, LX, SHORT, false, UNROLL, EPT>(k, bt, tl, perm, r2_s);
  else
    grid_tile<Lane, LX, SHORT, true, UNROLL, EPT>(k, bt, tl, perm, r2_s);
}

template <typename Lane, int LX, bool SHORT, int UNROLL, int EPT>
cudaError_t launch_grid(const BatchGroup& g, const BatchTensor* tensors, const BatchTile* tiles,
                        int* status, cudaStream_t s) {
  const uint32_t ntiles = g.end - g.begin;
  if (ntiles == 0) return cudaSuccess;
  relu_batch_grid_kernel<Lane, LX, SHORT, UNROLL, EPT>
      <<<ntiles, kBlock, 0, s>>>(g.k, tensors, tiles, g.begin, status);
  return cudaGetLastError();
}

template <typename Lane, int LX, bool SHORT, int UNROLL>
cudaError_t launch_persistent(const BatchGroup& g, const BatchTensor* tensors,
                              const BatchTile* tiles, unsigned int* counter, int* status,
                              int num_sms, int ctas_per_sm, cudaStream_t s) {
  auto kern = relu_batch_kernel<Lane, LX, SHORT, UNROLL>;
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

template <typename Lane, int LX, bool SHORT, int UNROLL>
cudaError_t launch_sched(const BatchGroup& g, const BatchTensor* tensors, const BatchTile* tiles,
                         unsigned int* counter, int* status, int num_sms,
                         const BatchLaunch& L, cudaStream_t s) {
  if (L.ctas_per_sm >= 0)
    return launch_persistent<Lane, LX, SHORT, UNROLL>(g, tensors, tiles, counter, status,
                                                      num_sms, L.ctas_per_sm, s);
  switch (L.elems_per_thread) {
    case 2: return launch_grid<Lane, LX, SHORT, UNROLL, 2>(g, tensors, tiles, status, s);
    case 4: return launch_grid<Lane, LX, SHORT, UNROLL, 4>(g, tensors, tiles, status, s);
    default: return launch_grid<Lane, LX, SHORT, UNROLL, 1>(g, tensors, tiles, status, s);
  }
}

// Key widths with every unroll variant.
template <typename Lane, int LX, bool SHORT>
cudaError_t launch_tuned(const BatchGroup& g, const BatchTensor* tensors, const BatchTile* tiles,
                         unsigned int* counter, int* status, int num_sms, const BatchLaunch& L,
                         cudaStream_t s) {
  switch (L.slot_unroll) {
    case 1:
      return launch_sched<Lane, LX, SHORT, 1>(g, tensors, tiles, counter, status, num_sms, L, s);
    case 2:
      return launch_sched<Lane, LX, SHORT, 2>(g, tensors, tiles, counter, status, num_sms, L, s);
    case 3:
      return launch_sched<Lane, LX, SHORT, 3>(g, tensors, tiles, counter, status, num_sms, L, s);
    default:
      return launch_sched<Lane, LX, SHORT, kSlotUnroll>(g, tensors, tiles, counter, status,
                                                        num_sms, L, s);
  }
}

// One thread per tile: the tile's tensor is the last one whose first tile is
// at or before it (binary search over the table; empty tensors own no tiles).
__global__ void __launch_bounds__(kBlock)
    expand_tiles_kernel(const BatchTensor* __restrict__ tensors, uint32_t count,
                        uint32_t ntiles, uint32_t tile, BatchTile* __restrict__ tiles) {
  const uint32_t w = blockIdx.x * kBlock + threadIdx.x;
  if (w >= ntiles) return;
  uint32_t lo = 0, hi = count;   // tensors[lo].first_tile <= w < tensors[hi].first_tile
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (tensors[mid].first_tile <= w) lo = mid;
    else hi = mid;
  }
  const uint64_t start = (uint64_t)(w - tensors[lo].first_tile) * tile;
  const uint64_t n = tensors[lo].n;
  BatchTile bt;
  bt.tensor = lo;
  bt.start = start;
  bt.count = (uint32_t)(n - start < (uint64_t)tile ? n - start : (uint64_t)tile);
  tiles[w] = bt;
}

}  // namespace

cudaError_t launch_expand_tiles(const BatchTensor* tensors, uint32_t count, uint32_t ntiles,
                                uint32_t tile, BatchTile* tiles, cudaStream_t s) {
  if (ntiles == 0 || count == 0) return cudaSuccess;
  expand_tiles_kernel<<<(ntiles + kBlock - 1) / kBlock, kBlock, 0, s>>>(tensors, count, ntiles,
                                                                        tile, tiles);
  return cudaGetLastError();
}

cudaError_t launch_relu_batch(const BatchTensor* tensors, const BatchTile* tiles,
                              const BatchGroup* groups, int ngroups, unsigned int* counters,
                              int* status, int num_sms, const BatchLaunch& L, cudaStream_t s) {
  for (int gi = 0; gi < ngroups; ++gi) {
    const BatchGroup& g = groups[gi];
    if (g.end <= g.begin) continue;
    unsigned int* ctr = counters + gi;
    cudaError_t e;
    if (g.k.ring_bits > 32) {
      if (g.k.lx == 24 && g.k.c + g.k.lx < 32)
        e = launch_tuned<uint64_t, 24, true>(g, tensors, tiles, ctr, status, num_sms, L, s);
      else
        e = launch_sched<uint64_t, 0, false, kSlotUnroll>(g, tensors, tiles, ctr, status, num_sms,
                                                          L, s);
    } else if (g.k.lx == 14) {
      e = launch_tuned<uint32_t, 14, false>(g, tensors, tiles, ctr, status, num_sms, L, s);
    } else if (g.k.lx == 9) {
      e = launch_tuned<uint32_t, 9, false>(g, tensors, tiles, ctr, status, num_sms, L, s);
    } else {
      e = launch_sched<uint32_t, 0, false, kSlotUnroll>(g, tensors, tiles, ctr, status, num_sms,
                                                        L, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bc
