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
//
// Every call looks up the array's device address on its device (the runtime
// gives it without allocating once the module is loaded, and a lookup per
// call stays right if the device's context was reset in between).  Calls on a
// stream that is being captured are refused: the tables are copied from host
// staging that the next call overwrites, so a replayed copy would read another
// call's tables.  bc_relu_batch_static_status reads the status word.
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
// since the source is pageable host memory) and the primes already checked.
// Guarded by one mutex.
std::mutex g_mu;
bc::BatchTensor g_host_tensors[BC_STATIC_MAX_TENSORS];
bc::BatchTile g_host_tiles[BC_STATIC_MAX_TILES];
bc::PrimeCache g_primes;
constexpr size_t kStatusOffset = 4 * bc::kMaxBatchGroups;

// Makes `device` current (restoring the caller's device on destruction).
struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == device || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceScope() {
    if (ok && prev >= 0) cudaSetDevice(prev);
  }
};

// Device address of g_batch_scratch on the current device (set-up of every
// call), or nullptr.
unsigned char* scratch_address() {
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_batch_scratch) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<unsigned char*>(addr);
}

// A stream in the middle of a capture (or one whose capture state cannot be
// read) is refused.
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace

extern "C" int bc_relu_batch_static(uint64_t seed, int device, void* cuda_stream,
                                    const bc_tensor_desc* descs, int count, int tile_elems) {
  if (count < 0 || (count > 0 && !descs) || device < 0) return BC_EINVAL;
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
  cudaStream_t s = (cudaStream_t)cuda_stream;

  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScope dev(device);
  if (!dev.ok) return BC_ECUDA;
  if (capturing(s)) return BC_EINVAL;
  unsigned char* base = scratch_address();   // set-up, with the device current
  if (!base) return BC_ECUDA;
  unsigned int* counters = reinterpret_cast<unsigned int*>(base);
  int* status = reinterpret_cast<int*>(base + kStatusOffset);
  bc::BatchTensor* d_tensors = reinterpret_cast<bc::BatchTensor*>(base + kHeaderBytes);
  bc::BatchTile* d_tiles = reinterpret_cast<bc::BatchTile*>(base + kHeaderBytes + kTensorBytes);

  const bc::RoundKeys rk = bc::make_round_keys(seed);
  // parameter groups of the batch (same l, lx, c, p); tiles of one group are
  // contiguous in the table
  int grp[BC_STATIC_MAX_TENSORS];
  bc::BatchGroup groups[bc::kMaxBatchGroups];
  int ngroups = 0;
  for (int t = 0; t < count; ++t) {
    const bc_tensor_desc& d = descs[t];
    bc::ReluConsts k;
    const int rc = bc::make_relu_consts(&d.params, rk, 0, g_primes, &k);
    if (rc != BC_OK) return rc;
    int g = 0;
    while (g < ngroups && !(groups[g].k.ring_bits == k.ring_bits && groups[g].k.lx == k.lx &&
                            groups[g].k.c == k.c && groups[g].k.mp.p == k.mp.p))
      ++g;
    if (g == ngroups) {
      if (ngroups == bc::kMaxBatchGroups) return BC_ELIMIT;
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
  size_t w = 0;
  for (int g = 0; g < ngroups; ++g) {
    groups[g].begin = (uint32_t)w;
    for (int t = 0; t < count; ++t) {
      if (grp[t] != g) continue;
      const uint64_t n = descs[t].n;
      for (uint64_t st = 0; st < n; st += tile) {
        g_host_tiles[w].tensor = (uint32_t)t;
        g_host_tiles[w].start = st;
        g_host_tiles[w].count = (uint32_t)(n - st < (uint64_t)tile ? n - st : (uint64_t)tile);
        ++w;
      }
    }
    groups[g].end = (uint32_t)w;
  }
  // counters and status word start at zero for every call, launched or not
  if (cudaMemsetAsync(base, 0, kHeaderBytes, s) != cudaSuccess) return BC_ECUDA;
  if (w == 0) return BC_OK;
  int num_sms = 1;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMemcpyAsync(d_tensors, g_host_tensors, sizeof(bc::BatchTensor) * count,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_tiles, g_host_tiles, sizeof(bc::BatchTile) * w, cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return BC_ECUDA;
  if (bc::launch_relu_batch(d_tensors, d_tiles, groups, ngroups, counters, status, num_sms,
                            bc::BatchLaunch{0, 1, 0}, s) != cudaSuccess)
    return BC_ECUDA;
  return BC_OK;
}

extern "C" int bc_relu_batch_static_status(int device, void* cuda_stream) {
  if (device < 0) return BC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScope dev(device);
  if (!dev.ok) return BC_ECUDA;
  if (capturing(s)) return BC_EINVAL;
  int st = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbolAsync(&st, g_batch_scratch, sizeof st, kStatusOffset,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_batch_scratch, &zero, sizeof zero, kStatusOffset,
                              cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BC_ECUDA;
  return st;
}
