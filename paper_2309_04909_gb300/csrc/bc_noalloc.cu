// Batched ReLU/DReLU for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: a plugin
// running inside a serving engine that owns every byte of device memory
// through its own pool, or a latency-critical loop in a process with a fixed
// memory budget, where cudaMalloc may fail or synchronise the device at the
// worst moment.  Such callers cannot even create a bc_ctx (bc_create reserves
// workspace).  bc_relu_batch_static serves them: it runs the same persistent
// tile-queue kernel as bc_relu_batch, but its scratch (the tensor table, the
// tile table, the work counter and the status word) lives in the fixed,
// file-scope device array below instead of memory the library allocates.
//
// The array is part of the loaded module, so every GPU that loads the library
// holds it (kStaticScratchBytes) until the process exits.  All calls share
// it and it keeps the last call's contents; the counter and the status word
// are cleared by every call before its launch.  Calls that overlap on the GPU
// (for example on two streams) race on the array.
#include <mutex>

#include "bc_internal.h"

namespace {

constexpr size_t kHeaderBytes = 256;   // work counters at 0 (one per group), status at 128
constexpr size_t kTensorBytes =
    ((BC_STATIC_MAX_TENSORS * sizeof(bc::BatchTensor) + 255) / 256) * 256;
constexpr size_t kTileBytes = ((BC_STATIC_MAX_TILES * sizeof(bc::BatchTile) + 255) / 256) * 256;
constexpr size_t kStaticScratchBytes = kHeaderBytes + kTensorBytes + kTileBytes;

static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

// Host-side staging of the tables (copied out before the copy call returns,
// since the source is pageable host memory) and the per-device address of
// g_batch_scratch.  Guarded by one mutex.
std::mutex g_mu;
bc::BatchTensor g_host_tensors[BC_STATIC_MAX_TENSORS];
bc::BatchTile g_host_tiles[BC_STATIC_MAX_TILES];
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

bool is_prime_u32(uint64_t q) {
  if (q < 2) return false;
  if (q % 2 == 0) return q == 2;
  for (uint64_t d = 3; d * d <= q; d += 2)
    if (q % d == 0) return false;
  return true;
}

// The constants of one tensor (same checks and values as the context path).
int static_consts(const bc_drelu_params* prm, uint32_t tensor_id, bc::ReluConsts* k) {
  const int ell = prm->ring_bits, lx = prm->lx, c = prm->key_off;
  if (ell < 2 || ell > 64 || lx < 1 || lx > 31 || c < 0 || c + 2 * lx > ell) return BC_EINVAL;
  const uint32_t p = prm->p ? prm->p : bc_prime_above(lx);
  const uint64_t lo = (uint64_t)1 << lx, hi = (uint64_t)1 << (lx + 1);
  if ((uint64_t)p <= lo || (uint64_t)p >= hi || !is_prime_u32(p)) return BC_EINVAL;
  uint32_t inv = p;
  for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
  const uint64_t r1 = ((uint64_t)1 << 32) % p;
  k->mp.p = p;
  k->mp.pinv = 0u - inv;
  k->mp.r2 = (uint32_t)((r1 * r1) % p);
  k->mp.pm1 = p - 1;
  k->ring_mask = ell >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << ell) - 1);
  k->ring_bits = (uint32_t)ell;
  k->lx = (uint32_t)lx;
  k->c = (uint32_t)c;
  k->mx = (uint32_t)(lo - 1);
  k->two_lx = (uint32_t)lo;
  k->p_minus_2lx = p - (uint32_t)lo;
  k->tensor_id = tensor_id;
  k->elem_base = 0;
  return BC_OK;
}

}  // namespace

extern "C" int bc_relu_batch_static(uint64_t seed, int device, void* cuda_stream,
                                    const bc_tensor_desc* descs, int count, int tile_elems) {
  if (count < 0 || (count > 0 && !descs) || device < 0 || device >= kMaxDevices) return BC_EINVAL;
  if (count > BC_STATIC_MAX_TENSORS) return BC_ELIMIT;
  const int tile = tile_elems > 0 ? tile_elems : 4096;
  if (tile > (1 << 30)) return BC_EINVAL;
  uint64_t ntiles = 0;
  for (int t = 0; t < count; ++t) {
    const bc_tensor_desc& d = descs[t];
    if (d.op != BC_OP_RELU && d.op != BC_OP_DRELU) return BC_EINVAL;
    if (d.n && (!d.sh0 || !d.sh1 || !d.o0 || !d.o1)) return BC_EINVAL;
    if (!bc::elem_range_ok(d.elem_offset, d.n)) return BC_EINVAL;
    ntiles += (d.n + tile - 1) / tile;
  }
  if (ntiles > BC_STATIC_MAX_TILES) return BC_ELIMIT;

  std::lock_guard<std::mutex> lock(g_mu);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return BC_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return BC_ECUDA;
  int rc = BC_OK;
  do {
    // set-up, once per device, with that device current
    if (!g_scratch_addr[device]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_batch_scratch) != cudaSuccess || !addr) {
        rc = BC_ECUDA;
        break;
      }
      g_scratch_addr[device] = static_cast<unsigned char*>(addr);
    }
    unsigned char* base = g_scratch_addr[device];
    unsigned int* counters = reinterpret_cast<unsigned int*>(base);
    int* status = reinterpret_cast<int*>(base + 4 * bc::kMaxBatchGroups);
    bc::BatchTensor* d_tensors = reinterpret_cast<bc::BatchTensor*>(base + kHeaderBytes);
    bc::BatchTile* d_tiles = reinterpret_cast<bc::BatchTile*>(base + kHeaderBytes + kTensorBytes);

    bc::RoundKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
      rk.k0[r] = k0;
      rk.k1[r] = k1;
      k0 += bc::kPhiloxW0;
      k1 += bc::kPhiloxW1;
    }
    // parameter groups of the batch (same l, lx, c, p); tiles of one group
    // are contiguous in the table
    int grp[BC_STATIC_MAX_TENSORS];
    bc::BatchGroup groups[bc::kMaxBatchGroups];
    int ngroups = 0;
    for (int t = 0; t < count && rc == BC_OK; ++t) {
      const bc_tensor_desc& d = descs[t];
      bc::ReluConsts k;
      rc = static_consts(&d.params, 0, &k);
      if (rc != BC_OK) break;
      k.rk = rk;
      int g = 0;
      while (g < ngroups && !(groups[g].k.ring_bits == k.ring_bits && groups[g].k.lx == k.lx &&
                              groups[g].k.c == k.c && groups[g].k.mp.p == k.mp.p))
        ++g;
      if (g == ngroups) {
        if (ngroups == bc::kMaxBatchGroups) {
          rc = BC_ELIMIT;
          break;
        }
        groups[ngroups].k = k;
        groups[ngroups].begin = groups[ngroups].end = 0;
        ++ngroups;
      }
      grp[t] = g;
      bc::BatchTensor& bt = g_host_tensors[t];
      bt.sh0 = d.sh0;
      bt.sh1 = d.sh1;
      bt.o0 = d.o0;
      bt.o1 = d.o1;
      bt.n = d.n;
      bt.tensor_id = d.tensor_id;
      bt.op = d.op;
      bt.elem_offset = d.elem_offset;
    }
    if (rc != BC_OK) break;
    size_t w = 0;
    for (int g = 0; g < ngroups; ++g) {
      groups[g].begin = (uint32_t)w;
      for (int t = 0; t < count; ++t) {
        if (grp[t] != g) continue;
        const uint64_t n = descs[t].n;
        for (uint64_t s = 0; s < n; s += tile) {
          g_host_tiles[w].tensor = (uint32_t)t;
          g_host_tiles[w].start = s;
          g_host_tiles[w].count = (uint32_t)(n - s < (uint64_t)tile ? n - s : (uint64_t)tile);
          ++w;
        }
      }
      groups[g].end = (uint32_t)w;
    }
    if (w == 0) break;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int num_sms = 1;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMemcpyAsync(d_tensors, g_host_tensors, sizeof(bc::BatchTensor) * count,
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_tiles, g_host_tiles, sizeof(bc::BatchTile) * w, cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemsetAsync(base, 0, kHeaderBytes, s) != cudaSuccess) {   // counters, status = 0
      rc = BC_ECUDA;
      break;
    }
    if (bc::launch_relu_batch(d_tensors, d_tiles, groups, ngroups, counters, status, num_sms,
                              bc::BatchLaunch{0, 1, 0}, s) != cudaSuccess)
      rc = BC_ECUDA;
  } while (0);
  if (prev != device) cudaSetDevice(prev);
  return rc;
}
