/*
 * bicoptor.h -- C-ABI of the GB300 Bicoptor 2.0 hot path.
 *
 * Paper: "Bicoptor 2.0: Addressing Challenges in Probabilistic Truncation for
 * Enhanced Privacy-Preserving Machine Learning" (arXiv 2309.04909).
 *
 * Three parties (P0, P1 holding 2-of-2 additive shares in Z_{2^l}, P2 the
 * helper; Sec. 2.1 "unbalanced mode") are simulated on one GPU.  Every step of
 * every party runs in this library's CUDA kernels; the messages the parties
 * would exchange are kept in registers (or written to audit buffers on
 * request) and their sizes are counted in bc_comm.
 *
 * Conventions for every entry point:
 *  - Share arrays are DEVICE pointers owned by the caller, except where an
 *    entry point's name ends in _host.  A ring element of Z_{2^l} is stored in
 *    a uint32_t lane when l <= 32 and a uint64_t lane when 32 < l <= 64, in
 *    canonical form (bits >= l are zero).  Inputs that are not canonical give
 *    undefined (but memory-safe) results; bc_set_checked makes calls refuse
 *    them.
 *  - Calls are asynchronous and ordered on the context's stream.  They return
 *    BC_OK (0) or a negative BC_E* code; on an error nothing is launched.
 *  - Hot calls allocate nothing: device workspace is reserved by bc_create
 *    and by bc_reserve.
 *  - Every entry point that launches work opens an NVTX range named after
 *    itself, so that a profiler timeline shows the calls.
 *  - Randomness: every pseudorandom value is Philox-4x32-10 keyed by the
 *    context seed, with the counter (element index, tensor_id, block,
 *    pair/purpose tag).  Results therefore depend only on (seed, tensor_id,
 *    element index, input), never on batch composition or launch shape.
 */
#ifndef BICOPTOR_H
#define BICOPTOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define BC_OK 0
#define BC_EINVAL (-1)   /* bad argument: sizes, parameters, NULL pointers      */
#define BC_ENOMEM (-2)   /* device workspace could not be reserved               */
#define BC_ECUDA (-3)    /* a CUDA call failed (see bc_last_cuda_error)          */
#define BC_ETIMEOUT (-4) /* a bounded device wait gave up (bc_parties_status)   */
#define BC_ECHECK (-5)   /* a device-side consistency check failed               */
#define BC_ELIMIT (-6)   /* request exceeds a fixed capacity (bc_relu_batch_static) */

typedef struct bc_ctx bc_ctx;

/* Parameters of Alg. drelu / Alg. relu (Sec. 5.4, key bits Sec. 6.1).
 *   ring_bits  l, 2..64
 *   lx         key bits, 1..31; the protocol works on lx+1 windows
 *   key_off    c >= 0, the lowest key bit; the window of step 3 for index i
 *              keeps bits c+i .. c+i+lx-1, so c + 2*lx <= l is required
 *   p          prime with 2^lx < p < 2^(lx+1) (Alg. modswitch needs
 *              log2 p = lx+1); 0 selects the smallest prime above 2^lx      */
typedef struct {
  int ring_bits;
  int lx;
  int key_off;
  uint32_t p;
} bc_drelu_params;

/* Protocol communication counted by the library, in BITS, summed over calls
 * since bc_create or bc_reset_comm.  A Z_p element counts ceil(log2 p) =
 * lx+1 bits, a ring element l bits (Table "compare": one-pass cost
 * (lx+1)*(lx+1) bits per sending party). */
typedef struct {
  uint64_t p0_to_p2, p1_to_p2;   /* masked, shuffled, reshared w (Alg. drelu step 8) */
  uint64_t p2_to_p0, p2_to_p1;   /* DReLU' reply (step 10) / e = DReLU' - b (Alg. relu) */
  uint64_t p0_to_p1, p1_to_p0;   /* Beaver openings d = x - a (and e for bc_mul_beaver) */
  uint64_t pre_p2_to_p1;         /* preprocessing: [c]_1 of the Beaver triple           */
  uint64_t rounds;               /* online communication rounds                        */
  uint64_t elements;             /* elements processed by interactive protocols        */
  uint64_t calls;                /* protocol calls                                     */
  uint64_t pre_p2_to_p0;         /* preprocessing: [s]_0 of the RSS protocol           */
  uint64_t rss_reshare;          /* replicated-product reshares P_i -> P_(i-1), all 3  */
} bc_comm;

/* Optional materialised messages of the next DReLU/ReLU calls (device
 * pointers, NULL = not wanted).  n elements, L = lx+1 slots:
 *   w0, w1      uint32 [n * L]  P0->P2 and P1->P2 messages, slot-major per element
 *   reply       lanes  [n]      P2->P1 [DReLU']_1 (drelu) or e (relu)
 *   open0/open1 lanes  [n]      P0->P1 / P1->P0 share of d = x - a (relu)
 *   pre_c1      lanes  [n]      P2->P1 preprocessing [c]_1 (relu)
 *   t, dprime   uint8  [n]      the flip bit and P2's DReLU'              */
typedef struct {
  uint32_t *w0, *w1;
  void *reply, *open0, *open1, *pre_c1;
  uint8_t *t, *dprime;
} bc_audit;

/* ---- context ------------------------------------------------------------ */

/* Create a context on `device` using `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  `seed` keys every pre-shared seed of the
 * simulation.  *out receives the context; free it with bc_destroy. */
int bc_create(bc_ctx **out, uint64_t seed, int device, void *cuda_stream);
int bc_destroy(bc_ctx *ctx);
int bc_set_stream(bc_ctx *ctx, void *cuda_stream);
int bc_synchronize(bc_ctx *ctx);
/* Checked mode (off by default; a debugging aid).  When on, every call that
 * takes device share arrays (and bc_relu_batch_plan, per tensor) first counts
 * on the GPU the input lanes that are not canonical (a bit at or above l set;
 * l = 32 and l = 64 lanes always are), waits for the count, and returns
 * BC_EINVAL without launching the operation if any lane fails.  The wait
 * makes every checked call synchronous with the context stream.
 * bc_linear_relu_host scans its host inputs on the host instead. */
int bc_set_checked(bc_ctx *ctx, int on);
const char *bc_strerror(int code);
/* Text of the last CUDA error seen by this context (empty if none). */
const char *bc_last_cuda_error(bc_ctx *ctx);

/* Smallest prime p with 2^lx < p < 2^(lx+1) (Alg. modswitch); 0 if lx is
 * outside 1..31. Host-only. */
uint32_t bc_prime_above(int lx);

/* ---- sharing (Sec. 2.2) ------------------------------------------------- */

/* Dealer: [x]_0 = x + R, [x]_1 = -R mod 2^l for fixed-point plaintexts
 * x (int64, device, n entries; reduced mod 2^l), R from the dealer stream of
 * (seed, tensor_id, element index).  Test/dealer utility, not a party's view. */
int bc_share(bc_ctx *ctx, int ring_bits, const int64_t *x, size_t n, uint32_t tensor_id,
             void *sh0, void *sh1);
/* x = [x]_0 + [x]_1 mod 2^l into lanes (device). */
int bc_reconstruct(bc_ctx *ctx, int ring_bits, const void *sh0, const void *sh1, size_t n,
                   void *x_out);

/* ---- non-interactive truncations and modulo switch ---------------------- */

/* Alg. smltrc (SecureML): P0 cut([x]_0, k) mod 2^l, P1 2^l - cut(2^l - [x]_1, k)
 * mod 2^l.  Outputs in Z_{2^l}.  0 <= k < l.  In-place allowed. */
int bc_trunc_prob(bc_ctx *ctx, int ring_bits, int k, const void *sh0, const void *sh1,
                  size_t n, void *o0, void *o1);
/* Alg. newtrc2 (Alg. newtrc when k2 = 0): keep bits k1 .. l-k2-1; outputs in
 * Z_{2^(l-k1-k2)} with that ring's lane width.  k1, k2 >= 0, k1 + k2 < l. */
int bc_trunc_det(bc_ctx *ctx, int ring_bits, int k1, int k2, const void *sh0, const void *sh1,
                 size_t n, void *o0, void *o1);
/* Alg. modswitch: shares in Z_{2^lp} (uint32 lanes, 1 <= lp <= 31) to shares
 * in Z_p (uint32), zero iff zero.  p prime, 2^lp < p < 2^32. */
int bc_mod_switch(bc_ctx *ctx, int lp, uint32_t p, const void *sh0, const void *sh1, size_t n,
                  uint32_t *o0, uint32_t *o1);

/* Alg. aby3trc (ABY3 probabilistic truncation, Sec. 2.4) between P0 and P1
 * with P2 dealing (r, r' = r / 2^k): [r]_0, [r']_0 from seed02, [r]_1 from
 * seed12, [r']_1 = r' - [r']_0 sent by P2 to P1; P0 and P1 open
 * alpha = x + r; P0 outputs alpha / 2^k - [r']_0, P1 outputs -[r']_1.  "/ 2^k"
 * is floor division of the two's-complement value.  fixed_r != 0 uses the
 * constant r = fixed_r (random shares) -- the implementation shortcut Sec. 4.1
 * shows hides e1.  Outputs in Z_{2^l}; 0 <= k < l. */
int bc_trunc_aby3(bc_ctx *ctx, int ring_bits, int k, const void *sh0, const void *sh1, size_t n,
                  uint32_t tensor_id, uint64_t fixed_r, void *o0, void *o1);

/* Alg. linear (truncate-then-multiply, Sec. 4.2): Alg. smltrc removes kx bits
 * from x and ky bits from y (kx + ky = the fractional bits; kx != ky for an odd
 * count), then the Beaver product of the truncated shares (triple as in
 * bc_mul_beaver for the same tensor_id).  One fused elementwise kernel. */
int bc_trunc_then_mul(bc_ctx *ctx, int ring_bits, int kx, int ky, const void *x0, const void *x1,
                      const void *y0, const void *y1, size_t n, uint32_t tensor_id, void *o0,
                      void *o1);

/* Beaver multiplication (Table "notation", Alg. relu preprocessing): the
 * triple comes from seed02/seed12, P2 sends [c]_1 to P1, d = x - a and
 * e = y - b are opened; [xy] = de + d[b] + e[a] + [c].  Exact in Z_{2^l}. */
int bc_mul_beaver(bc_ctx *ctx, int ring_bits, const void *x0, const void *x1, const void *y0,
                  const void *y1, size_t n, uint32_t tensor_id, void *o0, void *o1);

/* ---- DReLU / ReLU (Alg. drelu, Alg. relu) ------------------------------- */

/* Shares of DReLU(x) in Z_{2^l}: one fused kernel runs P0's and P1's steps
 * 1-8, P2's step 9 and the reply/unflip of steps 10-11 per element. */
int bc_drelu(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
             size_t n, uint32_t tensor_id, void *o0, void *o1);
/* Shares of ReLU(x) = x * DReLU(x) in Z_{2^l} via the seeded Beaver triple. */
int bc_relu(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
            size_t n, uint32_t tensor_id, void *o0, void *o1);

/* Materialise the messages of subsequent DReLU/ReLU calls into `bufs`
 * (NULL turns auditing off).  The buffers must hold the call's n elements. */
int bc_set_audit(bc_ctx *ctx, const bc_audit *bufs);

/* ---- RSS DReLU / ReLU (Alg. drelu2) ------------------------------------- */

/* 2-of-3 replicated shares in Z_{2^l}: component arrays x0, x1, x2 with
 * x = x0 + x1 + x2; P0 holds (x0, x1), P1 (x1, x2), P2 (x2, x0).  Outputs the
 * three components of [DReLU(x)] (bc_rss_drelu) or of [ReLU(x)] (bc_rss_relu,
 * the replicated product [x][DReLU]).  Preprocessing (replicated sharings of
 * t and of P2's bit s, [s xor t] by one replicated product) and Alg. drelu
 * between P0 ([x]_0 + [x]_1) and P1 ([x]_2) run in one fused kernel; P2
 * publishes d'' = s xor DReLU'. */
int bc_rss_drelu(bc_ctx *ctx, const bc_drelu_params *prm, const void *x0, const void *x1,
                 const void *x2, size_t n, uint32_t tensor_id, void *y0, void *y1, void *y2);
int bc_rss_relu(bc_ctx *ctx, const bc_drelu_params *prm, const void *x0, const void *x1,
                const void *x2, size_t n, uint32_t tensor_id, void *y0, void *y1, void *y2);

/* ---- the Bicoptor 1.0-style DReLU / ReLU (the baseline) ------------------ */

/* The protocol Bicoptor 2.0 improves on, as the paper describes it by
 * contrast (Table "compare"; Sec. "sub:cmp"; the notes on steps 3-4 of
 * Alg. drelu), for comparing communication and speed on the same GPU:
 * Alg. smltrc truncations in Z_{2^l} at key-bit positions c + i (i = 0..lx),
 * recursive sums S_i = sum_{k >= i} u_k with v_i = S_i - 1, masks by random
 * odd units r_k and reshares z_k in Z_{2^l}, P2's zero test in Z_{2^l}; the
 * flip, shuffle, reply and ReLU triple as in Bicoptor 2.0.  Each party sends
 * (lx+1) l bits per element (counted in bc_comm).  Needs c + lx < l; p is
 * ignored.  w0, w1 (optional, both or neither): the messages, n * (lx+1)
 * lanes each, slot-major per element.  Correct outside the SecureML
 * truncation's large-error events (probability |x| / 2^l per truncation),
 * which is what Alg. newtrc2 removes. */
int bc_drelu_b1(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
                size_t n, uint32_t tensor_id, void *o0, void *o1, void *w0, void *w1);
int bc_relu_b1(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
               size_t n, uint32_t tensor_id, void *o0, void *o1, void *w0, void *w1);

/* ---- party-separated DReLU / ReLU --------------------------------------- */

/* The message buffers of one party-separated call (device memory owned by
 * the caller).  Every message of Alg. drelu / Alg. relu lives here between
 * the sender's kernel and the receiver's:
 *   w0, w1      P0 -> P2 and P1 -> P2 (step 8), bc_party_msg_words(lx, n)
 *               uint32 words each, 16-byte aligned: the lx+1 values of lx+1
 *               bits per element, packed (groups of 32 elements; slot k of
 *               group g occupies the lx+1 words at (g * (lx+1) + k) * (lx+1),
 *               element 32g+l at bits [l (lx+1), (l+1)(lx+1)); the group
 *               count is ceil(n/32) rounded up to a multiple of 8)
 *   reply       lanes [n]: [DReLU']_1 to P1 (DReLU) / e = DReLU' - b (ReLU)
 *   open0/1     lanes [n]: P0 -> P1 and P1 -> P0 shares of d = x - a (ReLU)
 *   pre_c1      lanes [n]: P2 -> P1 preprocessing [c]_1 (ReLU)              */
typedef struct {
  uint32_t *w0, *w1;
  void *reply, *open0, *open1, *pre_c1;
} bc_party_msgs;

/* uint32 words of one packed w buffer for n elements: (lx+1)^2 bits per
 * element, n rounded up to a multiple of 256. */
size_t bc_party_msg_words(int lx, size_t n);

/* Alg. drelu / Alg. relu with each party's local work in its own kernel and
 * every message in `msgs`: P0 and P1 (steps 1-8, each expanding seed01
 * itself, + ReLU openings), then P2 (step 9, reply, [c]_1), then P0 and P1
 * finish.  Same outputs as bc_drelu / bc_relu and the same messages as their
 * audit buffers (unpacked). */
int bc_drelu_parties(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
                     size_t n, uint32_t tensor_id, void *o0, void *o1, const bc_party_msgs *msgs);
int bc_relu_parties(bc_ctx *ctx, const bc_drelu_params *prm, const void *sh0, const void *sh1,
                    size_t n, uint32_t tensor_id, void *o0, void *o1, const bc_party_msgs *msgs);
/* One party's stage of the same protocol, for callers that run P0, P1 and P2
 * as separate processes (each with its own context, possibly on its own GPU)
 * and move the messages between them (Alg. drelu steps 8-10, Alg. relu).
 * Every buffer is a device pointer in the memory of the party that runs the
 * stage; a message written by the sender's stage must be copied into the
 * receiver's buffer before the receiver's stage runs.  Layouts as in
 * bc_party_msgs (w: bc_party_msg_words(lx, n) words, 16-byte aligned for P2).
 *   bc_party_local   P0 (party 0) or P1 (party 1): steps 1-8 from its own share
 *                    [x]_party, expanding seed01 itself; writes its packed w
 *                    message to P2 and, for ReLU (relu != 0), its opening
 *                    [x]_party - [a]_party to the other party (`open`)
 *   bc_party_helper  P2: step 9 on both w messages; writes `reply` ([DReLU']_1
 *                    for P1 in DReLU, e = DReLU' - b for P0 and P1 in ReLU) and,
 *                    for ReLU, the preprocessing [c]_1 for P1 (`pre_c1`)
 *   bc_party_finish  P0 or P1: step 11 (DReLU: P0 needs no message, P1 the
 *                    reply) or the Beaver finish (ReLU: its own share, e,
 *                    both openings and, for P1, [c]_1); writes its output share
 * The outputs equal bc_drelu_parties / bc_relu_parties.  Each stage counts in
 * bc_comm the bits its party sends; P2's stage also counts the call's rounds,
 * elements and calls, so that the three contexts' counters add up to the
 * single-process call's. */
int bc_party_local(bc_ctx *ctx, int party, const bc_drelu_params *prm, int relu,
                   const void *share, size_t n, uint32_t tensor_id, uint32_t *w, void *open);
int bc_party_helper(bc_ctx *ctx, const bc_drelu_params *prm, int relu, size_t n,
                    uint32_t tensor_id, const uint32_t *w0, const uint32_t *w1, void *reply,
                    void *pre_c1);
int bc_party_finish(bc_ctx *ctx, int party, const bc_drelu_params *prm, int relu,
                    const void *share, size_t n, uint32_t tensor_id, const void *reply,
                    const void *open0, const void *open1, const void *pre_c1, void *out);

/* P2's kernel waits (at most 50 ms) for the bulk copies of its messages.
 * BC_OK, or BC_ETIMEOUT if that wait gave up in a party-separated call since
 * the last read (that call's outputs are then undefined).  Synchronises the
 * context's stream and clears the status. */
int bc_parties_status(bc_ctx *ctx);
/* Test hook for that bounded wait: while on (nonzero), P2's kernel issues no
 * copies, so its wait runs out after 1 ms and bc_parties_status reports
 * BC_ETIMEOUT.  Off by default; for tests only. */
int bc_test_drop_p2_copies(bc_ctx *ctx, int on);

int bc_get_comm(bc_ctx *ctx, bc_comm *out);
int bc_reset_comm(bc_ctx *ctx);

/* ---- batched ReLU over many tensors (persistent tile queue) -------------- */

#define BC_OP_RELU 0
#define BC_OP_DRELU 1

typedef struct {
  const void *sh0, *sh1;   /* input shares (lanes of params.ring_bits)   */
  void *o0, *o1;           /* output shares                              */
  uint64_t n;              /* elements                                   */
  uint32_t tensor_id;      /* keys the randomness of this tensor          */
  int op;                  /* BC_OP_RELU or BC_OP_DRELU                   */
  bc_drelu_params params;
  uint64_t elem_offset;    /* element index of sh0[0] within the tensor
                              `tensor_id` (a slice of a larger tensor gets
                              the randomness of those elements); usually 0.
                              elem_offset + n <= 2^48 (the Philox counter
                              holds 48 index bits), else BC_EINVAL */
} bc_tensor_desc;

/* Schedule of the batched launch (0 fields = library default).
 *   schedule          BC_SCHED_PERSISTENT: per parameter group, one persistent
 *                     grid whose warps take tiles from an atomic work counter;
 *                     BC_SCHED_GRID: one CTA per tile of 256 x elems_per_thread
 *                     elements (the hardware CTA scheduler is the queue;
 *                     tile_elems ignored)
 *   tile_elems        elements per queue tile (persistent schedule; default 512)
 *   ctas_per_sm       resident CTAs per SM of the persistent grid (0 = occupancy)
 *   elems_per_thread  grid schedule: 1, 2 or 4 elements per thread (default 1)
 *   slot_unroll       unroll of the per-element key-bit loop over the lx + 1
 *                     message slots: 1, 2 or 3, or 0 = the default, the whole
 *                     loop; honoured for lx = 24 at l = 64 and lx = 14, 9 at
 *                     l <= 32, other key widths run the loop unrolled by 2
 * Results do not depend on any of these (randomness is keyed by tensor id and
 * element index). Values out of range give BC_EINVAL. */
#define BC_SCHED_PERSISTENT 0
#define BC_SCHED_GRID 1
typedef struct {
  int tile_elems;
  int ctas_per_sm;
  int schedule;
  int elems_per_thread;
  int slot_unroll;
} bc_batch_config;

/* Plan a batch: group the tensors by parameters (l, lx, c, p; at most 32
 * groups), build the tile table on the host and copy it to device workspace
 * owned by the context (grown here, not in bc_relu_batch_run).  The plan
 * stays valid until the next bc_relu_batch_plan. */
int bc_relu_batch_plan(bc_ctx *ctx, const bc_tensor_desc *descs, int count,
                       const bc_batch_config *cfg);
/* Run the planned batch: one launch per parameter group (one launch for a
 * single-parameter batch), persistent or grid as planned.  Stream-capturable
 * (no host synchronisation inside). */
int bc_relu_batch_run(bc_ctx *ctx);
/* plan + run. */
int bc_relu_batch(bc_ctx *ctx, const bc_tensor_desc *descs, int count,
                  const bc_batch_config *cfg);
/* Status word of the last batched launch (BC_OK or BC_ECHECK);
 * synchronises the context's stream. */
int bc_batch_status(bc_ctx *ctx);

/* The batched DReLU/ReLU of bc_relu_batch (Alg. drelu / Alg. relu per tensor,
 * Sec. 6 per-network ReLU sets) on HOST buffers: sh0, sh1, o0 and o1 of every
 * descriptor are host pointers into page-locked memory mapped for the device
 * (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with the mapped flag;
 * a torch pin_memory() tensor qualifies).  The batched kernel loads the input
 * shares and stores the output shares across the host link itself, so no
 * device copy of the data is made; the tables are planned as by
 * bc_relu_batch_plan (into the context's workspace, replacing any earlier
 * plan).  Returns after the outputs are in host memory.  BC_EINVAL if a
 * buffer (n lanes of the descriptor's ring) is not mapped page-locked memory;
 * nothing is launched then.  Same results as bc_relu_batch on device copies. */
int bc_relu_batch_host(bc_ctx *ctx, const bc_tensor_desc *descs, int count,
                       const bc_batch_config *cfg);

/* Batched ReLU/DReLU that allocates nothing.  The paper has no counterpart:
 * this serves callers that may not call cudaMalloc -- code running inside a
 * host engine that owns all device memory through its own pool, or a loop
 * under a fixed memory budget where an allocation could fail or synchronise
 * the device.  Such callers cannot create a bc_ctx, so this entry point takes
 * the seed, device and stream directly.  It runs the same persistent
 * tile-queue kernel as bc_relu_batch (same results for the same seed) with its
 * scratch -- tensor table, tile table, work counter, status word -- in one
 * fixed file-scope device array of about 310 KB, which every GPU that loads
 * the library holds until the process exits.
 *   - At most BC_STATIC_MAX_TENSORS tensors and BC_STATIC_MAX_TILES tiles of
 *     `tile_elems` elements (0 = 4096) per call; larger requests return
 *     BC_ELIMIT before anything is launched.
 *   - Every call first looks up the array's device address on `device`, with
 *     that device current (its set-up; the runtime resolves the address of a
 *     loaded module without allocating).
 *   - A call on a stream that is being captured returns BC_EINVAL and does
 *     nothing: the tables are copied from host staging that the next call
 *     overwrites, so a captured copy would read another call's tables when
 *     replayed.
 *   - Calls share the array, which keeps the last call's contents; each call
 *     clears the counters and the status word before its launch.  Calls that
 *     overlap on the GPU (e.g. on two streams) race on the array.
 *   - The tables are copied from pageable host staging, which orders the copy
 *     after work already queued on `cuda_stream`.
 *   - No communication is counted (there is no context).
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
#define BC_STATIC_MAX_TENSORS 256
#define BC_STATIC_MAX_TILES 16384
int bc_relu_batch_static(uint64_t seed, int device, void *cuda_stream,
                         const bc_tensor_desc *descs, int count, int tile_elems);
/* Status word of the last bc_relu_batch_static launch on `device`: BC_OK, or
 * BC_ECHECK if the kernel met a tile that does not fit its tensor (what two
 * overlapping calls could leave in the shared tables) and skipped it.  Reads
 * and clears the word in stream order on `cuda_stream`, then synchronises
 * that stream; allocates nothing.  BC_EINVAL on a capturing stream. */
int bc_relu_batch_static_status(int device, void *cuda_stream);

/* ---- fused product -> truncation -> ReLU (Sec. 4, Alg. smltrc/newtrc, Alg. relu) */

typedef struct {
  int ring_bits;            /* l of x, y, the product and the ReLU           */
  int trunc_bits;           /* k removed after the product (2f -> f)          */
  bc_drelu_params relu;     /* ReLU parameters, relu.ring_bits == ring_bits   */
  const void *x0, *x1, *y0, *y1;
  size_t n;
  uint32_t tensor_id;       /* product uses tensor_id, ReLU tensor_id + 1     */
  void *prod0, *prod1;      /* product shares (l-bit lanes; optional)         */
  void *trc0, *trc1;        /* Alg. smltrc output (l-bit lanes; optional)     */
  void *det0, *det1;        /* Alg. newtrc output in Z_{2^(l-k)} (optional)   */
  void *relu0, *relu1;      /* ReLU of the probabilistically truncated product */
} bc_linear_relu_args;

/* One fused kernel per element: the Beaver product (Sec. 2.2) with the triple
 * of `tensor_id`, Alg. smltrc and Alg. newtrc (k1 = trunc_bits, k2 = 0) of the
 * product, and Alg. relu (tensor id tensor_id + 1) of the Alg. smltrc output.
 * Results equal bc_mul_beaver, bc_trunc_prob, bc_trunc_det and bc_relu called
 * in turn.  All pointers are device pointers.  x, y, relu are required;
 * prod, trc and det are optional in pairs (both NULL: not written; one NULL:
 * BC_EINVAL).  Communication is counted as for the product plus the ReLU. */
int bc_linear_relu(bc_ctx *ctx, const bc_linear_relu_args *a);

/* The same step with HOST pointers: x0,x1,y0,y1 in; relu0,relu1 and
 * optionally det0,det1 out (prod/trc fields are ignored).  Two paths:
 *   direct  every buffer is page-locked memory mapped for the device (from
 *           cudaHostAlloc/cudaMallocHost or cudaHostRegister): the fused
 *           kernel loads and stores it across the host link, one launch.
 *   staged  otherwise: chunks of bc_reserve's `chunk` elements are copied to
 *           device buffers, run and copied back, four chunks in flight on
 *           four streams so that both copy directions and the kernels of
 *           different chunks overlap (needs bc_reserve first, else BC_EINVAL).
 * bc_set_host_path chooses: BC_HOST_AUTO (direct when every buffer is mapped),
 * BC_HOST_DIRECT (BC_EINVAL if one is not), BC_HOST_STAGED.  Each host array
 * must hold n lanes: the direct path cannot check extents, and a short buffer
 * is an out-of-range device access.  Returns after the results are in host
 * memory. */
#define BC_HOST_AUTO 0
#define BC_HOST_DIRECT 1
#define BC_HOST_STAGED 2
int bc_linear_relu_host(bc_ctx *ctx, const bc_linear_relu_args *a);
int bc_set_host_path(bc_ctx *ctx, int path);
/* Set the chunk of the staged path to `chunk` elements, growing the device
 * staging (4 sets of 8 arrays of `chunk` 64-bit lanes) if needed. */
int bc_reserve(bc_ctx *ctx, size_t chunk);

/* ---- truncation-failure statistics (evaluation only) --------------------- */

/* Count elements whose reconstructed truncation differs from the plaintext
 * floor(x / 2^k) by more than one (the e1 failure of Sec. 3), given the
 * plaintext x (int64, device) and output shares in Z_{2^out_bits}.
 * *count (device uint64) is incremented. */
int bc_count_trunc_failures(bc_ctx *ctx, int out_bits, int k, const int64_t *x, const void *o0,
                            const void *o1, size_t n, unsigned long long *count);

/* ---- integer-pipe microbenchmarks (measuring aid) ------------------------ */

/* The paper has no counterpart: this measures, on `device`, the rates of the
 * integer instructions the hot path is bound by, for its roofline.  Each
 * kernel keeps 8 independent chains per thread over 8 CTAs of 256 threads per
 * SM (the widening products run as Philox-4x32 rounds, the hot path's form);
 * the best of three runs is reported, in warp-lane instructions per
 * second, plus the SM clock one CTA saw (cycle counter against the global
 * timer).  Allocates a few bytes and a stream, runs about 0.4 s, synchronises;
 * BC_ECUDA on a CUDA failure. */
typedef struct {
  double imad_wide_per_s;   /* 32x32->64 products, in Philox rounds          */
  double imad_per_s;        /* 32-bit multiply-adds                           */
  double alu_per_s;         /* integer-ALU instructions (xor, add pairs)      */
  double sm_mhz;            /* SM clock during the last run                   */
  int sm_count;
  double imad_hi_per_s;     /* high halves of 32x32 products (hi32(x*k))      */
} bc_int_peaks;
int bc_measure_int_peaks(int device, bc_int_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* BICOPTOR_H */
