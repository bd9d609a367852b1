// C-ABI of the library: context, argument checks, communication accounting,
// the batched tile planner, and host-buffer staging.  Every entry point is
// declared (with its citation) in include/bicoptor.h.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include <initializer_list>

#include <nvtx3/nvToolsExt.h>

#include "bc_internal.h"

struct bc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};   // more streams of the host staging
  uint64_t seed = 0;
  bc::RoundKeys rk{};
  int num_sms = 1;
  bc_comm comm{};
  bc::AuditPtrs audit{};
  char last_err[256] = {0};
  // validated (lx, p) pairs
  bc::PrimeCache primes;
  // batched launch plan
  bc::BatchTensor* d_tensors = nullptr;
  bc::BatchTile* d_tiles = nullptr;
  // pinned host staging of the tensor table, double-buffered: buffer i may be
  // refilled once the copy recorded by plan_ev[i] has finished
  bc::BatchTensor* h_tensors[2] = {nullptr, nullptr};
  cudaEvent_t plan_ev[2] = {nullptr, nullptr};
  bool plan_ev_live[2] = {false, false};
  int plan_next = 0;
  size_t cap_tensors = 0, cap_tiles = 0;
  unsigned int* d_counter = nullptr;     // one work counter per parameter group
  int* d_status = nullptr;
  uint32_t ntiles = 0;
  bc::BatchLaunch batch_launch{0, 1, 0};
  bc::BatchGroup groups[bc::kMaxBatchGroups];
  int ngroups = 0;
  bc_comm batch_comm{};                   // what one run of the plan adds
  bool planned = false;
  // host staging for bc_linear_relu_host: one set of chunk buffers per stream
  size_t stage_cap = 0;       // allocated elements per array
  size_t stage_chunk = 0;     // elements per chunk (<= stage_cap)
  void* stage[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;
  int host_path = BC_HOST_AUTO;
  // checked mode: canonical-form check of every input before a call
  bool checked = false;
  unsigned long long* d_check = nullptr;
  // party-separated calls: P2's wait status (sticky until read); test hook
  int* d_party_status = nullptr;
  bool drop_p2_copies = false;
};

namespace {

int cuda_fail(bc_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) snprintf(ctx->last_err, sizeof(ctx->last_err), "%s: %s", where, cudaGetErrorString(e));
  return BC_ECUDA;
}
// A named range on the NVTX timeline for the duration of an entry point
// (free when no profiler is attached).
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
};
#define BC_TRACE() Trace bc_trace_(__func__)

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

size_t lane_bytes(int bits) { return bits > 32 ? 8 : 4; }

using bc::is_prime_u32;
using bc::make_round_keys;
using bc::ring_mask;

// Checked mode: count, on the context stream, the lanes of the given arrays
// that have bits at or above ring_bits, wait, and refuse the call if any do.
int check_canonical(bc_ctx* ctx, int ring_bits, std::initializer_list<const void*> arrays,
                    size_t n) {
  if (!ctx->checked || n == 0 || ring_bits == 32 || ring_bits == 64) return BC_OK;
  CK(cudaMemsetAsync(ctx->d_check, 0, sizeof(unsigned long long), ctx->stream));
  for (const void* a : arrays)
    if (a) CK(bc::launch_count_noncanonical(ring_bits, a, n, ctx->d_check, ctx->num_sms,
                                            ctx->stream));
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_check, sizeof bad, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return bad ? BC_EINVAL : BC_OK;
}

// Checks of Alg. drelu's parameters; fills the kernel constants.
int make_consts(bc_ctx* ctx, const bc_drelu_params* prm, uint32_t tensor_id,
                bc::ReluConsts* k) {
  return bc::make_relu_consts(prm, ctx->rk, tensor_id, ctx->primes, k);
}

// Communication of one protocol call over n elements (bits).
void add_comm(bc_comm* c, const bc_comm& d) {
  c->p0_to_p2 += d.p0_to_p2;
  c->p1_to_p2 += d.p1_to_p2;
  c->p2_to_p0 += d.p2_to_p0;
  c->p2_to_p1 += d.p2_to_p1;
  c->p0_to_p1 += d.p0_to_p1;
  c->p1_to_p0 += d.p1_to_p0;
  c->pre_p2_to_p1 += d.pre_p2_to_p1;
  c->rounds += d.rounds;
  c->elements += d.elements;
  c->calls += d.calls;
  c->pre_p2_to_p0 += d.pre_p2_to_p0;
  c->rss_reshare += d.rss_reshare;
}

bc_comm relu_comm(int ell, int lx, uint64_t n, bool relu) {
  bc_comm d{};
  const uint64_t L = (uint64_t)lx + 1, zp_bits = (uint64_t)lx + 1;   // ceil(log2 p) = lx + 1
  d.p0_to_p2 = n * L * zp_bits;    // Alg. drelu step 8
  d.p1_to_p2 = n * L * zp_bits;
  if (relu) {
    d.p2_to_p0 = n * (uint64_t)ell;      // e = DReLU' - b
    d.p2_to_p1 = n * (uint64_t)ell;
    d.p0_to_p1 = n * (uint64_t)ell;      // share of d = x - a
    d.p1_to_p0 = n * (uint64_t)ell;
    d.pre_p2_to_p1 = n * (uint64_t)ell;  // [c]_1
  } else {
    d.p2_to_p1 = n * (uint64_t)ell;      // [DReLU']_1 (P0's share comes from seed02)
  }
  d.rounds = n ? 2 : 0;
  d.elements = n;
  d.calls = 1;
  return d;
}

bc_comm mul_comm(int ell, uint64_t n) {
  bc_comm d{};
  d.p0_to_p1 = 2 * n * (uint64_t)ell;   // shares of d = x - a and e = y - b
  d.p1_to_p0 = 2 * n * (uint64_t)ell;
  d.pre_p2_to_p1 = n * (uint64_t)ell;   // [c]_1
  d.rounds = n ? 1 : 0;
  d.elements = n;
  d.calls = 1;
  return d;
}

int run_relu(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1, size_t n,
             uint32_t tensor_id, void* o0, void* o1, bool relu, uint64_t elem_base,
             cudaStream_t s, bool count) {
  if (!ctx) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  bc::ReluConsts k;
  int rc = make_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  if (s == ctx->stream && (rc = check_canonical(ctx, prm->ring_bits, {sh0, sh1}, n))) return rc;
  k.elem_base = elem_base;
  if (n) CK(bc::launch_relu(k, relu, sh0, sh1, n, o0, o1, ctx->audit, ctx->num_sms, s));
  if (count) add_comm(&ctx->comm, relu_comm(prm->ring_bits, prm->lx, n, relu));
  return BC_OK;
}

}  // namespace

extern "C" {

const char* bc_strerror(int code) {
  switch (code) {
    case BC_OK: return "ok";
    case BC_EINVAL: return "invalid argument";
    case BC_ENOMEM: return "out of device memory";
    case BC_ECUDA: return "CUDA error";
    case BC_ETIMEOUT: return "bounded device wait timed out";
    case BC_ECHECK: return "device consistency check failed";
    default: return "unknown error";
  }
}

const char* bc_last_cuda_error(bc_ctx* ctx) { return ctx ? ctx->last_err : ""; }

uint32_t bc_prime_above(int lx) {
  if (lx < 1 || lx > 31) return 0;
  // trial division takes microseconds at lx = 24 and every call with p = 0
  // asks, so each lx is searched once (a racing second search stores the
  // same value)
  static std::atomic<uint32_t> found[32];
  const uint32_t known = found[lx].load(std::memory_order_relaxed);
  if (known) return known;
  uint64_t q = ((uint64_t)1 << lx) + 1;
  while (!is_prime_u32(q)) ++q;
  found[lx].store((uint32_t)q, std::memory_order_relaxed);
  return (uint32_t)q;
}

int bc_create(bc_ctx** out, uint64_t seed, int device, void* cuda_stream) {
  if (!out) return BC_EINVAL;
  *out = nullptr;
  bc_ctx* ctx = new bc_ctx();
  ctx->device = device;
  ctx->seed = seed;
  ctx->rk = make_round_keys(seed);
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counter, sizeof(unsigned int) * bc::kMaxBatchGroups);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_check, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_party_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_party_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&ctx->plan_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    int rc = (e == cudaErrorMemoryAllocation) ? BC_ENOMEM : BC_ECUDA;
    bc_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return BC_OK;
}

int bc_destroy(bc_ctx* ctx) {
  if (!ctx) return BC_EINVAL;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < 3; ++i) {
    if (ctx->aux[i]) {
      cudaStreamSynchronize(ctx->aux[i]);
      cudaStreamDestroy(ctx->aux[i]);
    }
  }
  cudaFree(ctx->d_tensors);
  cudaFree(ctx->d_tiles);
  for (int i = 0; i < 2; ++i) {
    cudaFreeHost(ctx->h_tensors[i]);
    if (ctx->plan_ev[i]) cudaEventDestroy(ctx->plan_ev[i]);
  }
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_check);
  cudaFree(ctx->d_party_status);
  for (int i = 0; i < 4; ++i) cudaFree(ctx->stage[i]);
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  delete ctx;
  return BC_OK;
}

int bc_set_stream(bc_ctx* ctx, void* cuda_stream) {
  if (!ctx) return BC_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return BC_OK;
}

int bc_synchronize(bc_ctx* ctx) {
  if (!ctx) return BC_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  return BC_OK;
}

int bc_share(bc_ctx* ctx, int ring_bits, const int64_t* x, size_t n, uint32_t tensor_id,
             void* sh0, void* sh1) {
  if (!ctx || ring_bits < 1 || ring_bits > 64) return BC_EINVAL;
  if (n && (!x || !sh0 || !sh1)) return BC_EINVAL;
  BC_TRACE();
  CK(bc::launch_share(ring_bits, ctx->rk, x, n, tensor_id, 0, sh0, sh1, ctx->num_sms, ctx->stream));
  return BC_OK;
}

int bc_reconstruct(bc_ctx* ctx, int ring_bits, const void* sh0, const void* sh1, size_t n,
                   void* x_out) {
  if (!ctx || ring_bits < 1 || ring_bits > 64) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !x_out)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {sh0, sh1}, n)) return rc;
  CK(bc::launch_reconstruct(ring_bits, sh0, sh1, n, x_out, ctx->num_sms, ctx->stream));
  return BC_OK;
}

int bc_trunc_prob(bc_ctx* ctx, int ring_bits, int k, const void* sh0, const void* sh1, size_t n,
                  void* o0, void* o1) {
  if (!ctx || ring_bits < 1 || ring_bits > 64 || k < 0 || k >= ring_bits) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {sh0, sh1}, n)) return rc;
  CK(bc::launch_trunc_prob(ring_bits, k, sh0, sh1, n, o0, o1, ctx->num_sms, ctx->stream));
  return BC_OK;
}

int bc_trunc_det(bc_ctx* ctx, int ring_bits, int k1, int k2, const void* sh0, const void* sh1,
                 size_t n, void* o0, void* o1) {
  if (!ctx || ring_bits < 1 || ring_bits > 64 || k1 < 0 || k2 < 0 || k1 + k2 >= ring_bits)
    return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  // outputs of a narrower lane than the inputs must not alias them
  if (lane_bytes(ring_bits) != lane_bytes(ring_bits - k1 - k2) && (o0 == sh0 || o1 == sh1))
    return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {sh0, sh1}, n)) return rc;
  CK(bc::launch_trunc_det(ring_bits, k1, k2, sh0, sh1, n, o0, o1, ctx->num_sms, ctx->stream));
  return BC_OK;
}

int bc_mod_switch(bc_ctx* ctx, int lp, uint32_t p, const void* sh0, const void* sh1, size_t n,
                  uint32_t* o0, uint32_t* o1) {
  if (!ctx || lp < 1 || lp > 31) return BC_EINVAL;
  if ((uint64_t)p <= ((uint64_t)1 << lp) || !is_prime_u32(p)) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, lp, {sh0, sh1}, n)) return rc;
  CK(bc::launch_mod_switch(lp, p, sh0, sh1, n, o0, o1, ctx->num_sms, ctx->stream));
  return BC_OK;
}

int bc_mul_beaver(bc_ctx* ctx, int ring_bits, const void* x0, const void* x1, const void* y0,
                  const void* y1, size_t n, uint32_t tensor_id, void* o0, void* o1) {
  if (!ctx || ring_bits < 1 || ring_bits > 64) return BC_EINVAL;
  if (n && (!x0 || !x1 || !y0 || !y1 || !o0 || !o1)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {x0, x1, y0, y1}, n)) return rc;
  CK(bc::launch_mul_beaver(ring_bits, ctx->rk, x0, x1, y0, y1, n, tensor_id, 0, o0, o1,
                           ctx->num_sms, ctx->stream));
  add_comm(&ctx->comm, mul_comm(ring_bits, n));
  return BC_OK;
}

int bc_trunc_aby3(bc_ctx* ctx, int ring_bits, int k, const void* sh0, const void* sh1, size_t n,
                  uint32_t tensor_id, uint64_t fixed_r, void* o0, void* o1) {
  if (!ctx || ring_bits < 2 || ring_bits > 64 || k < 0 || k >= ring_bits) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {sh0, sh1}, n)) return rc;
  CK(bc::launch_trunc_aby3(ring_bits, ctx->rk, k, sh0, sh1, n, tensor_id,
                           fixed_r & ring_mask(ring_bits), o0, o1, ctx->num_sms, ctx->stream));
  bc_comm d{};
  d.p0_to_p1 = d.p1_to_p0 = n * (uint64_t)ring_bits;   // shares of alpha = x + r
  d.pre_p2_to_p1 = n * (uint64_t)ring_bits;            // [r']_1
  d.rounds = n ? 1 : 0;
  d.elements = n;
  d.calls = 1;
  add_comm(&ctx->comm, d);
  return BC_OK;
}

int bc_trunc_then_mul(bc_ctx* ctx, int ring_bits, int kx, int ky, const void* x0, const void* x1,
                      const void* y0, const void* y1, size_t n, uint32_t tensor_id, void* o0,
                      void* o1) {
  if (!ctx || ring_bits < 1 || ring_bits > 64 || kx < 0 || ky < 0 || kx >= ring_bits ||
      ky >= ring_bits)
    return BC_EINVAL;
  if (n && (!x0 || !x1 || !y0 || !y1 || !o0 || !o1)) return BC_EINVAL;
  BC_TRACE();
  if (int rc = check_canonical(ctx, ring_bits, {x0, x1, y0, y1}, n)) return rc;
  CK(bc::launch_trunc_then_mul(ring_bits, ctx->rk, kx, ky, x0, x1, y0, y1, n, tensor_id, o0, o1,
                               ctx->num_sms, ctx->stream));
  add_comm(&ctx->comm, mul_comm(ring_bits, n));
  return BC_OK;
}

int bc_drelu(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1, size_t n,
             uint32_t tensor_id, void* o0, void* o1) {
  BC_TRACE();
  return run_relu(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, false, 0, ctx ? ctx->stream : nullptr,
                  true);
}

int bc_relu(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1, size_t n,
            uint32_t tensor_id, void* o0, void* o1) {
  BC_TRACE();
  return run_relu(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, true, 0, ctx ? ctx->stream : nullptr,
                  true);
}

int bc_set_audit(bc_ctx* ctx, const bc_audit* b) {
  if (!ctx) return BC_EINVAL;
  ctx->audit = bc::AuditPtrs{};
  if (b) {
    ctx->audit.w0 = b->w0;
    ctx->audit.w1 = b->w1;
    ctx->audit.reply = b->reply;
    ctx->audit.open0 = b->open0;
    ctx->audit.open1 = b->open1;
    ctx->audit.pre_c1 = b->pre_c1;
    ctx->audit.t = b->t;
    ctx->audit.dprime = b->dprime;
  }
  return BC_OK;
}

static int run_rss(bc_ctx* ctx, const bc_drelu_params* prm, const void* x0, const void* x1,
                   const void* x2, size_t n, uint32_t tensor_id, void* y0, void* y1, void* y2,
                   bool relu) {
  if (!ctx) return BC_EINVAL;
  if (n && (!x0 || !x1 || !x2 || !y0 || !y1 || !y2)) return BC_EINVAL;
  bc::ReluConsts k;
  int rc = make_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  BC_TRACE();
  if ((rc = check_canonical(ctx, prm->ring_bits, {x0, x1, x2}, n))) return rc;
  const void* x[3] = {x0, x1, x2};
  void* y[3] = {y0, y1, y2};
  if (n) CK(bc::launch_rss(k, relu, x, n, y, ctx->stream));
  const uint64_t ell = (uint64_t)prm->ring_bits, L = (uint64_t)prm->lx + 1;
  bc_comm d{};
  d.p0_to_p2 = d.p1_to_p2 = n * L * L;        // Alg. drelu step 8
  d.p2_to_p0 = d.p2_to_p1 = n;                // the public bit d''
  d.pre_p2_to_p0 = n * ell;                   // [s]_0
  d.rss_reshare = 3 * n * ell * (relu ? 2 : 1);   // [s][t] (and [x][DReLU])
  d.rounds = n ? (relu ? 3 : 2) : 0;
  d.elements = n;
  d.calls = 1;
  add_comm(&ctx->comm, d);
  return BC_OK;
}

int bc_rss_drelu(bc_ctx* ctx, const bc_drelu_params* prm, const void* x0, const void* x1,
                 const void* x2, size_t n, uint32_t tensor_id, void* y0, void* y1, void* y2) {
  return run_rss(ctx, prm, x0, x1, x2, n, tensor_id, y0, y1, y2, false);
}

int bc_rss_relu(bc_ctx* ctx, const bc_drelu_params* prm, const void* x0, const void* x1,
                const void* x2, size_t n, uint32_t tensor_id, void* y0, void* y1, void* y2) {
  return run_rss(ctx, prm, x0, x1, x2, n, tensor_id, y0, y1, y2, true);
}

size_t bc_party_msg_words(int lx, size_t n) {
  if (lx < 1 || lx > 31) return 0;
  return (size_t)bc::party_msg_words((uint32_t)lx, n);
}

static int run_parties(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
                       size_t n, uint32_t tensor_id, void* o0, void* o1,
                       const bc_party_msgs* m, bool relu) {
  if (!ctx || !m) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1 || !m->w0 || !m->w1 || !m->reply)) return BC_EINVAL;
  if (n && relu && (!m->open0 || !m->open1 || !m->pre_c1)) return BC_EINVAL;
  // P2 fetches the packed messages with bulk copies: 16-byte aligned buffers
  if (n && ((((uintptr_t)m->w0) | ((uintptr_t)m->w1)) & 15u)) return BC_EINVAL;
  bc::ReluConsts k;
  int rc = make_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  BC_TRACE();
  if ((rc = check_canonical(ctx, prm->ring_bits, {sh0, sh1}, n))) return rc;
  if (n)
    CK(bc::launch_parties(k, relu, sh0, sh1, n, o0, o1, m->w0, m->w1, m->open0, m->open1,
                          m->reply, m->pre_c1, ctx->d_party_status, ctx->drop_p2_copies,
                          ctx->stream));
  add_comm(&ctx->comm, relu_comm(prm->ring_bits, prm->lx, n, relu));
  return BC_OK;
}

int bc_drelu_parties(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
                     size_t n, uint32_t tensor_id, void* o0, void* o1, const bc_party_msgs* m) {
  return run_parties(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, m, false);
}

int bc_relu_parties(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
                    size_t n, uint32_t tensor_id, void* o0, void* o1, const bc_party_msgs* m) {
  return run_parties(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, m, true);
}

// ---- the Bicoptor 1.0-style DReLU / ReLU ---------------------------------------

static int run_b1(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
                  size_t n, uint32_t tensor_id, void* o0, void* o1, void* w0, void* w1,
                  bool relu) {
  if (!ctx || !prm) return BC_EINVAL;
  const int ell = prm->ring_bits, lx = prm->lx, c = prm->key_off;
  if (ell < 2 || ell > 64 || lx < 1 || lx > 31 || c < 0 || c + lx >= ell) return BC_EINVAL;
  if (n && (!sh0 || !sh1 || !o0 || !o1)) return BC_EINVAL;
  if (!w0 != !w1) return BC_EINVAL;
  BC_TRACE();
  int rc;
  if ((rc = check_canonical(ctx, ell, {sh0, sh1}, n))) return rc;
  bc::ReluConsts k{};
  k.rk = ctx->rk;
  k.ring_mask = ring_mask(ell);
  k.ring_bits = (uint32_t)ell;
  k.lx = (uint32_t)lx;
  k.c = (uint32_t)c;
  k.tensor_id = tensor_id;
  k.elem_base = 0;
  if (n) CK(bc::launch_b1(k, relu, sh0, sh1, n, o0, o1, w0, w1, ctx->stream));
  bc_comm d = relu_comm(ell, lx, n, relu);
  d.p0_to_p2 = d.p1_to_p2 = (uint64_t)n * (uint64_t)(lx + 1) * (uint64_t)ell;   // ring elements
  add_comm(&ctx->comm, d);
  return BC_OK;
}

int bc_drelu_b1(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
                size_t n, uint32_t tensor_id, void* o0, void* o1, void* w0, void* w1) {
  return run_b1(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, w0, w1, false);
}

int bc_relu_b1(bc_ctx* ctx, const bc_drelu_params* prm, const void* sh0, const void* sh1,
               size_t n, uint32_t tensor_id, void* o0, void* o1, void* w0, void* w1) {
  return run_b1(ctx, prm, sh0, sh1, n, tensor_id, o0, o1, w0, w1, true);
}

// ---- one party's stage --------------------------------------------------------

static int stage_consts(bc_ctx* ctx, const bc_drelu_params* prm, uint32_t tensor_id,
                        bc::ReluConsts* k) {
  if (!ctx) return BC_EINVAL;
  return make_consts(ctx, prm, tensor_id, k);
}

int bc_party_local(bc_ctx* ctx, int party, const bc_drelu_params* prm, int relu,
                   const void* share, size_t n, uint32_t tensor_id, uint32_t* w, void* open) {
  bc::ReluConsts k;
  int rc = stage_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  if (party != 0 && party != 1) return BC_EINVAL;
  if (n && (!share || !w || (relu && !open))) return BC_EINVAL;
  BC_TRACE();
  if ((rc = check_canonical(ctx, prm->ring_bits, {share}, n))) return rc;
  bc::PartyIo io{};
  io.sh[party] = share;
  io.w[party] = w;
  io.open[party] = open;
  if (n)
    CK(bc::launch_party_stage(k, relu != 0, 1, party, io, n, ctx->d_party_status,
                              ctx->drop_p2_copies, ctx->stream));
  const bc_comm full = relu_comm(prm->ring_bits, prm->lx, n, relu != 0);
  bc_comm mine{};
  (party == 0 ? mine.p0_to_p2 : mine.p1_to_p2) = full.p0_to_p2;
  if (relu) (party == 0 ? mine.p0_to_p1 : mine.p1_to_p0) = full.p0_to_p1;
  add_comm(&ctx->comm, mine);
  return BC_OK;
}

int bc_party_helper(bc_ctx* ctx, const bc_drelu_params* prm, int relu, size_t n,
                    uint32_t tensor_id, const uint32_t* w0, const uint32_t* w1, void* reply,
                    void* pre_c1) {
  bc::ReluConsts k;
  int rc = stage_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  if (n && (!w0 || !w1 || !reply || (relu && !pre_c1))) return BC_EINVAL;
  // P2 fetches the packed messages with bulk copies: 16-byte aligned buffers
  if (n && ((((uintptr_t)w0) | ((uintptr_t)w1)) & 15u)) return BC_EINVAL;
  BC_TRACE();
  bc::PartyIo io{};
  io.w[0] = const_cast<uint32_t*>(w0);
  io.w[1] = const_cast<uint32_t*>(w1);
  io.reply = reply;
  io.pre_c1 = pre_c1;
  if (n)
    CK(bc::launch_party_stage(k, relu != 0, 2, 2, io, n, ctx->d_party_status,
                              ctx->drop_p2_copies, ctx->stream));
  const bc_comm full = relu_comm(prm->ring_bits, prm->lx, n, relu != 0);
  bc_comm mine{};
  mine.p2_to_p0 = full.p2_to_p0;
  mine.p2_to_p1 = full.p2_to_p1;
  mine.pre_p2_to_p1 = full.pre_p2_to_p1;
  mine.rounds = full.rounds;     // the call's rounds, elements and calls are counted once,
  mine.elements = full.elements; // by P2, so that the three parties' counters add up to
  mine.calls = full.calls;       // the single-process call's
  add_comm(&ctx->comm, mine);
  return BC_OK;
}

int bc_party_finish(bc_ctx* ctx, int party, const bc_drelu_params* prm, int relu,
                    const void* share, size_t n, uint32_t tensor_id, const void* reply,
                    const void* open0, const void* open1, const void* pre_c1, void* out) {
  bc::ReluConsts k;
  int rc = stage_consts(ctx, prm, tensor_id, &k);
  if (rc) return rc;
  if (party != 0 && party != 1) return BC_EINVAL;
  if (n && !out) return BC_EINVAL;
  if (n && !relu && party == 1 && !reply) return BC_EINVAL;
  if (n && relu && (!share || !reply || !open0 || !open1 || (party == 1 && !pre_c1)))
    return BC_EINVAL;
  BC_TRACE();
  bc::PartyIo io{};
  io.sh[party] = share;
  io.out[party] = out;
  io.open[0] = const_cast<void*>(open0);
  io.open[1] = const_cast<void*>(open1);
  io.reply = const_cast<void*>(reply);
  io.pre_c1 = const_cast<void*>(pre_c1);
  if (n)
    CK(bc::launch_party_stage(k, relu != 0, 3, party, io, n, ctx->d_party_status,
                              ctx->drop_p2_copies, ctx->stream));
  return BC_OK;
}

int bc_parties_status(bc_ctx* ctx) {
  if (!ctx) return BC_EINVAL;
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->d_party_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_party_status, 0, sizeof(int), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return st;
}

int bc_test_drop_p2_copies(bc_ctx* ctx, int on) {
  if (!ctx) return BC_EINVAL;
  ctx->drop_p2_copies = on != 0;
  return BC_OK;
}

int bc_get_comm(bc_ctx* ctx, bc_comm* out) {
  if (!ctx || !out) return BC_EINVAL;
  *out = ctx->comm;
  return BC_OK;
}

int bc_reset_comm(bc_ctx* ctx) {
  if (!ctx) return BC_EINVAL;
  ctx->comm = bc_comm{};
  return BC_OK;
}

// ---- batched launch -------------------------------------------------------

int bc_relu_batch_plan(bc_ctx* ctx, const bc_tensor_desc* descs, int count,
                       const bc_batch_config* cfg) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return BC_EINVAL;
  const bool grid_sched = cfg && cfg->schedule == BC_SCHED_GRID;
  if (cfg && cfg->schedule != BC_SCHED_GRID && cfg->schedule != BC_SCHED_PERSISTENT)
    return BC_EINVAL;
  const int ept = cfg && cfg->elems_per_thread > 0 ? cfg->elems_per_thread : 1;
  const int unroll = cfg ? cfg->slot_unroll : 0;
  if ((grid_sched && ept != 1 && ept != 2 && ept != 4) || unroll < 0 || unroll > 3)
    return BC_EINVAL;
  const int tile = grid_sched ? bc::kBlock * ept
                              : (cfg && cfg->tile_elems > 0) ? cfg->tile_elems : 512;
  if (tile > (1 << 30)) return BC_EINVAL;
  // persistent: CTAs per SM (0 = occupancy); grid schedule: -1
  const int per_sm = grid_sched ? -1 : (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm : 0;
  std::vector<bc::BatchTensor> tens((size_t)count);
  std::vector<int> grp((size_t)count);
  bc::BatchGroup groups[bc::kMaxBatchGroups];
  int ngroups = 0;
  size_t ntiles = 0;
  bc_comm add{};
  for (int t = 0; t < count; ++t) {
    const bc_tensor_desc& d = descs[t];
    if (d.op != BC_OP_RELU && d.op != BC_OP_DRELU) return BC_EINVAL;
    if (d.n && (!d.sh0 || !d.sh1 || !d.o0 || !d.o1)) return BC_EINVAL;
    if (!bc::elem_range_ok(d.elem_offset, d.n)) return BC_EINVAL;
    bc::ReluConsts k;
    int rc = make_consts(ctx, &d.params, 0, &k);
    if (rc) return rc;
    if ((rc = check_canonical(ctx, d.params.ring_bits, {d.sh0, d.sh1}, d.n))) return rc;
    int g = 0;
    while (g < ngroups && !(groups[g].k.ring_bits == k.ring_bits && groups[g].k.lx == k.lx &&
                            groups[g].k.c == k.c && groups[g].k.mp.p == k.mp.p))
      ++g;
    if (g == ngroups) {
      if (ngroups == bc::kMaxBatchGroups) return BC_EINVAL;   // too many parameter sets
      groups[ngroups].k = k;
      groups[ngroups].begin = groups[ngroups].end = 0;
      ++ngroups;
    }
    grp[t] = g;
    tens[t].sh0 = d.sh0;
    tens[t].sh1 = d.sh1;
    tens[t].o0 = d.o0;
    tens[t].o1 = d.o1;
    tens[t].n = d.n;
    tens[t].tensor_id = d.tensor_id;
    tens[t].op = d.op;
    tens[t].elem_offset = d.elem_offset;
    ntiles += (d.n + tile - 1) / tile;
    add_comm(&add, relu_comm(d.params.ring_bits, d.params.lx, d.n, d.op == BC_OP_RELU));
  }
  if (ntiles > 0xFFFFFFF0u) return BC_EINVAL;
  add.rounds = count ? 2 : 0;   // all tensors share the two rounds of one batched call
  add.calls = count ? 1 : 0;
  if ((size_t)count > ctx->cap_tensors || ntiles > ctx->cap_tiles) {
    // growing: everything queued that may read the old tables must finish
    CK(cudaStreamSynchronize(ctx->stream));
    const size_t capt = std::max<size_t>(std::max<size_t>(count, 64), ctx->cap_tensors);
    const size_t capl = std::max<size_t>(std::max<size_t>(ntiles, 1024), ctx->cap_tiles);
    cudaFree(ctx->d_tensors);
    cudaFree(ctx->d_tiles);
    ctx->d_tensors = nullptr;
    ctx->d_tiles = nullptr;
    for (int i = 0; i < 2; ++i) {
      cudaFreeHost(ctx->h_tensors[i]);
      ctx->h_tensors[i] = nullptr;
      ctx->plan_ev_live[i] = false;
    }
    ctx->cap_tensors = ctx->cap_tiles = 0;
    bool ok = cudaMalloc(&ctx->d_tensors, capt * sizeof(bc::BatchTensor)) == cudaSuccess &&
              cudaMalloc(&ctx->d_tiles, capl * sizeof(bc::BatchTile)) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
      ok = cudaMallocHost(&ctx->h_tensors[i], capt * sizeof(bc::BatchTensor)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return BC_ENOMEM;
    }
    ctx->cap_tensors = capt;
    ctx->cap_tiles = capl;
  }
  // this plan's staging buffer: wait only for ITS previous copy to finish
  const int sb = ctx->plan_next;
  if (ctx->plan_ev_live[sb]) CK(cudaEventSynchronize(ctx->plan_ev[sb]));
  bc::BatchTensor* h_tensors = ctx->h_tensors[sb];
  // Tensors grouped by parameter group; within a group the largest come first
  // so that the long ones start early and short ones fill the tail.  The
  // table holds them in that order with the index of each one's first tile;
  // the tile table itself is written on the device.
  std::vector<int> order(count);
  for (int t = 0; t < count; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return grp[a] != grp[b] ? grp[a] < grp[b] : descs[a].n > descs[b].n;
  });
  uint32_t w = 0;
  for (int oi = 0; oi < count; ++oi) {
    const int t = order[oi];
    if (oi == 0 || grp[order[oi - 1]] != grp[t]) groups[grp[t]].begin = w;
    h_tensors[oi] = tens[t];
    h_tensors[oi].first_tile = w;
    w += (uint32_t)((descs[t].n + tile - 1) / tile);
    groups[grp[t]].end = w;
  }
  // Stream order puts the copy and the expansion after every kernel already
  // queued, so a batch still running keeps reading the previous tables until
  // it is done.
  if (count)
    CK(cudaMemcpyAsync(ctx->d_tensors, h_tensors, sizeof(bc::BatchTensor) * count,
                       cudaMemcpyHostToDevice, ctx->stream));
  CK(bc::launch_expand_tiles(ctx->d_tensors, (uint32_t)count, w, (uint32_t)tile, ctx->d_tiles,
                             ctx->stream));
  CK(cudaEventRecord(ctx->plan_ev[sb], ctx->stream));
  ctx->plan_ev_live[sb] = true;
  ctx->plan_next = sb ^ 1;
  for (int g = 0; g < ngroups; ++g) ctx->groups[g] = groups[g];
  ctx->ngroups = ngroups;
  ctx->ntiles = (uint32_t)w;
  ctx->batch_launch = bc::BatchLaunch{per_sm, grid_sched ? ept : 1, unroll};
  ctx->batch_comm = add;
  ctx->planned = true;
  return BC_OK;
}

int bc_relu_batch_run(bc_ctx* ctx) {
  if (!ctx || !ctx->planned) return BC_EINVAL;
  BC_TRACE();
  CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int) * bc::kMaxBatchGroups, ctx->stream));
  CK(bc::launch_relu_batch(ctx->d_tensors, ctx->d_tiles, ctx->groups, ctx->ngroups,
                           ctx->d_counter, ctx->d_status, ctx->num_sms, ctx->batch_launch,
                           ctx->stream));
  add_comm(&ctx->comm, ctx->batch_comm);
  return BC_OK;
}

int bc_relu_batch(bc_ctx* ctx, const bc_tensor_desc* descs, int count, const bc_batch_config* cfg) {
  int rc = bc_relu_batch_plan(ctx, descs, count, cfg);
  if (rc) return rc;
  return bc_relu_batch_run(ctx);
}

int bc_batch_status(bc_ctx* ctx) {
  if (!ctx) return BC_EINVAL;
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return st;
}

}  // extern "C"

namespace {

// Device address of a host pointer that the GPU can load from and store to
// (page-locked memory of the CUDA allocator or registered with it), else NULL.
void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Driver query of a pointer's allocation, reached through the runtime's entry
// point table (no link-time dependence on the driver library): memory type,
// device address and the extent of the allocation it belongs to.
typedef int (*PointerGetAttributesFn)(unsigned int, int*, void**, unsigned long long);
PointerGetAttributesFn pointer_query() {
  static PointerGetAttributesFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttributes", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PointerGetAttributesFn>(f);
  }();
  return fn;
}

// Device addresses of many host pointers.  The pointers of a batch are mostly
// slices of a few large page-locked allocations, so each allocation is looked
// up once: the driver reports the allocation's extent with its device address,
// and every later buffer that lies inside a known allocation maps by the same
// offset without another query.  Without the extent (an older driver), each
// buffer's first and last byte are checked separately.
struct HostMap {
  struct Span {
    uintptr_t lo, hi;   // host range [lo, hi) of one mapped allocation
    intptr_t delta;     // device address - host address
  };
  std::vector<Span> spans;
  void* map(const void* p, size_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    for (const Span& s : spans)
      if (a >= s.lo && a + bytes <= s.hi) return reinterpret_cast<void*>(a + s.delta);
    if (PointerGetAttributesFn q = pointer_query()) {
      // CU_POINTER_ATTRIBUTE_MEMORY_TYPE (2), _DEVICE_POINTER (3),
      // _RANGE_START_ADDR (11), _RANGE_SIZE (12); CU_MEMORYTYPE_HOST = 1
      int attrs[4] = {2, 3, 11, 12};
      unsigned int type = 0;
      unsigned long long dptr = 0, start = 0;
      size_t size = 0;
      void* data[4] = {&type, &dptr, &start, &size};
      if (q(4, attrs, data, (unsigned long long)a) == 0 && type == 1 && dptr && size &&
          start <= a && a - start < size) {
        const Span s{(uintptr_t)start, (uintptr_t)start + size, (intptr_t)dptr - (intptr_t)a};
        spans.push_back(s);
        return a + bytes <= s.hi ? reinterpret_cast<void*>(a + s.delta) : nullptr;
      }
    }
    void* d = mapped_host(p);
    if (!d) return nullptr;
    // the last byte must belong to the same mapping (same offset)
    if (bytes > 1 && mapped_host(static_cast<const char*>(p) + bytes - 1) !=
                         static_cast<char*>(d) + bytes - 1)
      return nullptr;
    spans.push_back({a, a + bytes, reinterpret_cast<intptr_t>(d) - (intptr_t)a});
    return d;
  }
};

}  // namespace

extern "C" {

int bc_relu_batch_host(bc_ctx* ctx, const bc_tensor_desc* descs, int count,
                       const bc_batch_config* cfg) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return BC_EINVAL;
  if (count == 0) return BC_OK;
  BC_TRACE();
  std::vector<bc_tensor_desc> dev(descs, descs + count);
  HostMap hm;
  for (bc_tensor_desc& d : dev) {
    if (d.n == 0) continue;
    if (d.params.ring_bits < 2 || d.params.ring_bits > 64) return BC_EINVAL;
    const size_t bytes = d.n * lane_bytes(d.params.ring_bits);
    const void* in[2] = {d.sh0, d.sh1};
    void* out[2] = {d.o0, d.o1};
    for (int q = 0; q < 2; ++q) {
      if (!in[q] || !out[q]) return BC_EINVAL;
      in[q] = hm.map(in[q], bytes);
      out[q] = hm.map(out[q], bytes);
      if (!in[q] || !out[q]) return BC_EINVAL;   // not page-locked mapped memory
    }
    d.sh0 = in[0];
    d.sh1 = in[1];
    d.o0 = out[0];
    d.o1 = out[1];
  }
  int rc = bc_relu_batch_plan(ctx, dev.data(), count, cfg);
  if (rc) return rc;
  if ((rc = bc_relu_batch_run(ctx))) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return BC_OK;
}

// ---- product -> truncations -> ReLU ---------------------------------------

namespace {

int check_linear(const bc_linear_relu_args* a) {
  if (!a) return BC_EINVAL;
  if (a->ring_bits < 2 || a->ring_bits > 64 || a->relu.ring_bits != a->ring_bits) return BC_EINVAL;
  if (a->trunc_bits < 0 || a->trunc_bits >= a->ring_bits) return BC_EINVAL;
  return BC_OK;
}

// The fused step kernel over n elements starting at element `base`; prod/trc/
// det pointers may be NULL (not written).
int linear_relu_device(bc_ctx* ctx, const bc_linear_relu_args* a, const bc::LinearIo& io,
                       size_t n, uint64_t base, cudaStream_t s) {
  bc::LinearConsts c;
  int rc = make_consts(ctx, &a->relu, a->tensor_id + 1, &c.k);
  if (rc) return rc;
  c.k.elem_base = base;
  c.mul_tid = a->tensor_id;
  c.trunc = (uint32_t)a->trunc_bits;
  c.det_mask = ring_mask(a->ring_bits - a->trunc_bits);
  c.det_wide = a->ring_bits - a->trunc_bits > 32 ? 1u : 0u;
  if (n) CK(bc::launch_linear_relu(c, io, n, s));
  return BC_OK;
}

// Checked mode on host buffers: every lane of the n-lane array below 2^ring_bits
// (scanned where the data lives, before anything is copied or launched).
bool host_canonical(const void* a, size_t n, int ring_bits) {
  if (ring_bits == 32 || ring_bits == 64) return true;
  if (ring_bits < 32) {
    const uint32_t* v = static_cast<const uint32_t*>(a);
    for (size_t i = 0; i < n; ++i)
      if (v[i] >> ring_bits) return false;
  } else {
    const uint64_t* v = static_cast<const uint64_t*>(a);
    for (size_t i = 0; i < n; ++i)
      if (v[i] >> ring_bits) return false;
  }
  return true;
}


}  // namespace

int bc_linear_relu(bc_ctx* ctx, const bc_linear_relu_args* a) {
  if (!ctx) return BC_EINVAL;
  int rc = check_linear(a);
  if (rc) return rc;
  if (a->n && (!a->x0 || !a->x1 || !a->y0 || !a->y1 || !a->relu0 || !a->relu1)) return BC_EINVAL;
  if (!a->prod0 != !a->prod1 || !a->trc0 != !a->trc1 || !a->det0 != !a->det1) return BC_EINVAL;
  BC_TRACE();
  if ((rc = check_canonical(ctx, a->ring_bits, {a->x0, a->x1, a->y0, a->y1}, a->n))) return rc;
  const bc::LinearIo io{a->x0, a->x1, a->y0, a->y1, a->prod0, a->prod1, a->trc0,
                        a->trc1, a->det0, a->det1, a->relu0, a->relu1};
  rc = linear_relu_device(ctx, a, io, a->n, 0, ctx->stream);
  if (rc) return rc;
  add_comm(&ctx->comm, mul_comm(a->ring_bits, a->n));
  add_comm(&ctx->comm, relu_comm(a->ring_bits, a->relu.lx, a->n, true));
  return BC_OK;
}

int bc_set_checked(bc_ctx* ctx, int on) {
  if (!ctx) return BC_EINVAL;
  ctx->checked = on != 0;
  return BC_OK;
}

int bc_set_host_path(bc_ctx* ctx, int path) {
  if (!ctx || path < BC_HOST_AUTO || path > BC_HOST_STAGED) return BC_EINVAL;
  ctx->host_path = path;
  return BC_OK;
}

int bc_reserve(bc_ctx* ctx, size_t max_chunk) {
  if (!ctx || max_chunk == 0) return BC_EINVAL;
  if (max_chunk > ctx->stage_cap) {
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 3; ++i) CK(cudaStreamSynchronize(ctx->aux[i]));
    for (int i = 0; i < 4; ++i) {
      cudaFree(ctx->stage[i]);
      ctx->stage[i] = nullptr;
    }
    ctx->stage_cap = ctx->stage_chunk = 0;
    const size_t per = ((max_chunk * 8 + 255) / 256) * 256;   // one 64-bit array, 256 B aligned
    for (int i = 0; i < 4; ++i) {
      if (cudaMalloc(&ctx->stage[i], per * 8) != cudaSuccess) {
        cudaGetLastError();
        return BC_ENOMEM;
      }
    }
    ctx->stage_cap = max_chunk;
  }
  ctx->stage_chunk = max_chunk;
  return BC_OK;
}

int bc_linear_relu_host(bc_ctx* ctx, const bc_linear_relu_args* a) {
  if (!ctx) return BC_EINVAL;
  int rc = check_linear(a);
  if (rc) return rc;
  if (a->n && (!a->x0 || !a->x1 || !a->y0 || !a->y1 || !a->relu0 || !a->relu1)) return BC_EINVAL;
  if (!a->det0 != !a->det1) return BC_EINVAL;
  const bool det = a->det0 != nullptr;
  if (a->n == 0) return BC_OK;
  BC_TRACE();
  if (ctx->checked)
    for (const void* h : {a->x0, a->x1, a->y0, a->y1})
      if (!host_canonical(h, a->n, a->ring_bits)) return BC_EINVAL;
  // direct path: every buffer is mapped page-locked memory, so the fused
  // kernel loads the inputs and stores the outputs across the host link
  const void* hp[8] = {a->x0, a->x1, a->y0, a->y1, a->relu0, a->relu1, a->det0, a->det1};
  void* dp[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool direct = ctx->host_path != BC_HOST_STAGED;
  for (int q = 0; q < (det ? 8 : 6) && direct; ++q)
    direct = (dp[q] = mapped_host(hp[q])) != nullptr;
  if (direct) {
    const bc::LinearIo io{dp[0], dp[1], dp[2], dp[3], nullptr, nullptr, nullptr,
                          nullptr, dp[6], dp[7], dp[4], dp[5]};
    rc = linear_relu_device(ctx, a, io, a->n, 0, ctx->stream);
    if (rc) return rc;
  } else {
    if (ctx->host_path == BC_HOST_DIRECT) return BC_EINVAL;   // some buffer is not mapped
    if (ctx->stage_chunk == 0) return BC_EINVAL;
    const size_t lb = lane_bytes(a->ring_bits);
    const size_t db = lane_bytes(a->ring_bits - a->trunc_bits);
    const size_t per = ((ctx->stage_cap * 8 + 255) / 256) * 256;
    const size_t chunk = ctx->stage_chunk;
    cudaStream_t st[4] = {ctx->stream, ctx->aux[0], ctx->aux[1], ctx->aux[2]};
    // the other streams start after everything queued on the context stream
    CK(cudaEventRecord(ctx->ev_start, ctx->stream));
    for (int i = 0; i < 3; ++i) CK(cudaStreamWaitEvent(ctx->aux[i], ctx->ev_start, 0));
    // chunk j runs on stream j % 4 with stage set j % 4: copies in, the fused
    // kernel, copies out; four chunks in flight let the two copy directions
    // and the kernels of different chunks overlap
    size_t j = 0;
    for (size_t off = 0; off < a->n; off += chunk, ++j) {
      const size_t m = std::min(chunk, a->n - off);
      cudaStream_t s = st[j % 4];
      char* base = static_cast<char*>(ctx->stage[j % 4]);
      void* b[8];
      for (int q = 0; q < 8; ++q) b[q] = base + per * q;
      for (int q = 0; q < 4; ++q)
        CK(cudaMemcpyAsync(b[q], static_cast<const char*>(hp[q]) + off * lb, m * lb,
                           cudaMemcpyHostToDevice, s));
      const bc::LinearIo io{b[0], b[1], b[2], b[3], nullptr, nullptr, nullptr,
                            nullptr, det ? b[6] : nullptr, det ? b[7] : nullptr, b[4], b[5]};
      rc = linear_relu_device(ctx, a, io, m, off, s);
      if (rc) return rc;
      for (int q = 4; q < (det ? 8 : 6); ++q) {
        const size_t w = q < 6 ? lb : db;
        CK(cudaMemcpyAsync(static_cast<char*>(const_cast<void*>(hp[q])) + off * w, b[q], m * w,
                           cudaMemcpyDeviceToHost, s));
      }
    }
    for (int i = 0; i < 3; ++i) CK(cudaStreamSynchronize(ctx->aux[i]));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  add_comm(&ctx->comm, mul_comm(a->ring_bits, a->n));
  add_comm(&ctx->comm, relu_comm(a->ring_bits, a->relu.lx, a->n, true));
  return BC_OK;
}

int bc_count_trunc_failures(bc_ctx* ctx, int out_bits, int k, const int64_t* x, const void* o0,
                            const void* o1, size_t n, unsigned long long* count) {
  if (!ctx || out_bits < 1 || out_bits > 64 || k < 0 || k > 63 || !count) return BC_EINVAL;
  if (n && (!x || !o0 || !o1)) return BC_EINVAL;
  CK(bc::launch_count_failures(out_bits, k, x, o0, o1, n, count, ctx->num_sms, ctx->stream));
  return BC_OK;
}

}  // extern "C"
