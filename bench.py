"""Benchmark of the Bicoptor 2.0 hot path on GB300.

Default workload (one "step" = every ReLU tensor of one batch through the
whole protocol): the ReLU set of a ResNet-18-shaped CNN on 224x224x3 inputs,
32 images, once in Z_{2^64} (f = 16, lx = 24 key bits, c = 0) and once more
in Z_{2^32} (f = 12, (lx, c) = (14, 4)) -- 1,088 tensors, 147,718,144
elements, Laplace(0, 2) activations -- as one CUDA-graph-captured batched
launch per parameter group.  Three parties simulated on one GPU; input shares
resident in HBM.  The fused step of a linear layer at l = 64 (Beaver product
-> SecureML and deterministic truncation -> ReLU, 2^22 elements) and the other
workloads are reported beside it.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ReLU elems/s on 1 GB300 (3 parties sim.), % roofline, batched vs plain; p99 ms"
# headline: the ResNet-18 224x224 ReLU set in both rings
RESNET_IMAGES = 32
WORKLOAD = ("ResNet-18 224x224 ReLU set x{images} images, once in Z_2^64 (f=16, lx=24, c=0) "
            "and once in Z_2^32 (f=12, lx=14, c=4): {tensors} tensors, {elems} elements, "
            "Laplace(0, 2) activations; one CUDA-graph-captured batched launch per parameter "
            "group")
BASE_SEED = 0xB1C0_2309_0490_9000
# DRAM bytes per element of the batched kernel over both rings: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the two launches of one step
# of a 4-image set (354.5 MB), divided by its 18,464,768 elements
TRAFFIC_PER_ELEM_BATCH = 19.20
# the fused step of a linear layer (reported beside the headline)
FUSED_WORKLOAD = ("Z_2^64 f=16 Beaver product of 2^22 Gaussian(sigma=4) share pairs -> "
                  "trunc k=16 (SecureML prob + det) -> ReLU lx=24 c=0 of the prob-truncated "
                  "product")
N_DEFAULT = 1 << 22
RING, FRAC, K_TRUNC, LX, KEY_OFF = 64, 16, 16, 24, 0
SEED = 1
# DRAM bytes per element of the fused step kernel: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of one 2^21-element launch (90.42 MB) / its elements
TRAFFIC_PER_ELEM = 43.11


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="resnet18",
                    choices=["resnet18", "fused", "b1-pair", "parties3"],
                    help="resnet18: the batched ReLU set (default, the headline); fused: the "
                         "fused linear-layer step alone (for profiling, with --step); b1-pair: "
                         "one Bicoptor 1.0-style DReLU and one Bicoptor 2.0 DReLU launch on the "
                         "same --n shares at l = 64, lx = 24 (for profiling); parties3: the "
                         "ReLU of --n elements with P0, P1 and P2 as three processes on GPU 0, "
                         "messages through host memory (gloo), per-party compute and transport "
                         "time")
    ap.add_argument("--party-transport", default="ipc", choices=["ipc", "gloo"],
                    help="with --workload parties3 -- ipc: each message copied by the GPU into "
                         "the receiver's own device buffer (CUDA IPC), token handshake over "
                         "gloo; gloo: messages through host memory")
    ap.add_argument("--images", type=int, default=RESNET_IMAGES,
                    help="images of the ResNet-18 set (32 in the workload; fewer for profiling)")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--fused-steps", type=int, default=1000,
                    help="timed steps of the fused linear-layer step")
    ap.add_argument("--step", default="fused", choices=["fused", "chain", "parties", "rss"],
                    help="with --workload fused -- fused: one kernel per step; chain: the same "
                         "step as four launches (product, two truncations, ReLU) through HBM, "
                         "each timed; parties / rss: the ReLU of the step's truncated product "
                         "by the party-separated launches / the RSS protocol")
    ap.add_argument("--no-autotune", action="store_true",
                    help="run the headline in the default launch shape (grid, 256-element "
                         "tiles, one element per thread, the key-bit loop unrolled whole), which "
                         "the autotuner keeps unless another beats it by more than 1%%, without "
                         "timing the others first (for profiling: no other launches precede the "
                         "step's)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the headline alone (for profiling): skip e2e, the CPU "
                         "baseline, the multiplier microbenchmark and every extra")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window of the offered-load serving run (the full trace is "
                         "60 s); the 90%% and 50%% load points use --serve-load-seconds")
    ap.add_argument("--serve-load-seconds", type=float, default=8.0)
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving trace at the offered 2,000 req/s and print it")
    return ap.parse_args()


def workload_inputs(n: int, seed: int = SEED):
    from paper_2309_04909_gb300 import workloads as W
    X = W.gaussian_reals(n, 4.0, seed=seed, stream=0)
    Y = W.gaussian_reals(n, 4.0, seed=seed, stream=1)
    xi = np.rint(np.ldexp(X, FRAC)).astype(np.int64)
    yi = np.rint(np.ldexp(Y, FRAC)).astype(np.int64)
    return xi, yi


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_chain(xi, yi, seed, threads):
    """The oracle's run of one step over a sample (first elements)."""
    import oracle as O
    n = xi.size
    idx = np.arange(n, dtype=np.uint64)
    x0, x1 = O.share(RING, xi.astype(np.uint64), seed, 1, idx=idx)
    y0, y1 = O.share(RING, yi.astype(np.uint64), seed, 2, idx=idx)
    p0, p1 = O.mul_beaver(RING, x0, x1, y0, y1, seed, 3, idx=idx)
    t0, t1 = O.trunc_prob(RING, K_TRUNC, p0, p1)
    O.trunc_det(RING, K_TRUNC, 0, p0, p1)
    O.relu(O.params(RING, LX, KEY_OFF), t0, t1, seed, 4, idx=idx, threads=threads)


def cpu_rate(n_target_s: float, xi, yi, threads):
    """Time the oracle on a sample sized for about n_target_s seconds."""
    m = 2048
    t0 = time.perf_counter()
    oracle_chain(xi[:m], yi[:m], 77, threads)
    dt = time.perf_counter() - t0
    per = dt / m
    m2 = int(min(xi.size, max(m, n_target_s / per)))
    t0 = time.perf_counter()
    oracle_chain(xi[:m2], yi[:m2], 77, threads)
    dt = time.perf_counter() - t0
    return m2 / dt, m2, dt


def cpu_configs(threads: int, min_elems: int = 10_000_000):
    """The oracle's ReLU (OpenMP over `threads` cores) on at least `min_elems`
    elements of the batched workloads, extrapolated linearly to their full
    size: the VGG-16 32x32 set of 128 images (l = 64, lx = 24, c = 0) and both
    rings of the ResNet-18 224x224 set of 32 images (l = 64; l = 32 with
    lx = 14, c = 4)."""
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    out = {}

    def sample(ts, ring, frac, full):
        xs, m = [], 0
        for r, rb in zip(ts.reals, ts.ring_bits):
            if rb != ring:
                continue
            xs.append(np.rint(np.ldexp(r, frac)).astype(np.int64))
            m += r.size
            if m >= min_elems:
                break
        x = np.concatenate(xs)
        return x, full

    # the first images of each set are the same as in the full batch (per-image
    # streams), so only as many images as the sample needs are generated
    per_vgg, per_res = sum(W.VGG16_32_LAYERS), sum(W.RESNET18_224_LAYERS)
    vgg = W.vgg16_batch(-(-min_elems // per_vgg), seed=2)
    res = W.resnet18_mixed_batch(-(-min_elems // per_res), seed=3)
    for name, ts, ring, frac, lx, c, full in (
            ("vgg16_l64", vgg, 64, 16, 24, 0, 128 * per_vgg),
            ("resnet18_l64", res, 64, 16, 24, 0, 32 * per_res),
            ("resnet18_l32", res, 32, 12, 14, 4, 32 * per_res)):
        x, full = sample(ts, ring, frac, full)
        idx = np.arange(x.size, dtype=np.uint64)
        s0, s1 = O.share(ring, (x.astype(np.uint64) & np.uint64((1 << ring) - 1)
                                if ring < 64 else x.astype(np.uint64)), 9, 1, idx=idx)
        t0 = time.perf_counter()
        O.relu(O.params(ring, lx, c), s0, s1, 9, 2, idx=idx, threads=threads)
        dt = time.perf_counter() - t0
        out[name] = {"elems_per_s": x.size / dt, "sample_elems": int(x.size), "seconds": dt,
                     "full_elems": int(full), "full_seconds_extrapolated": full * dt / x.size}
    out["cores"] = threads
    return out


def run_reference(args):
    """The reference arm: the CPU oracle on the headline's workload.  Each step
    runs the oracle's ReLU on the first m elements of each ring's part of the
    ResNet-18 set (whole tensors in order, with the tensor ids and shares of
    the GPU run), m sized so that warm-up and timed steps take about two
    minutes on all host cores."""
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    from paper_2309_04909_gb300.replicas import rank_seed
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = O.max_threads()
    O.set_threads(0)
    seed = rank_seed(BASE_SEED, 0)
    ts = W.resnet18_mixed_batch(1, seed=3)        # image 0 of the set (per-image streams)
    per_img = len(W.RESNET18_224_LAYERS)
    parts = []
    for s_idx, (ring, frac, lx, c) in enumerate(((64, 16, 24, 0), (32, 12, 14, 4))):
        idx = [i for i in range(len(ts.sizes)) if ts.ring_bits[i] == ring]
        x = np.concatenate([np.rint(np.ldexp(ts.reals[i], frac)).astype(np.int64) for i in idx])
        mask = np.uint64((1 << ring) - 1) if ring < 64 else np.uint64(2**64 - 1)
        s0, s1 = O.share(ring, x.astype(np.uint64) & mask, seed, 30 + ring)
        spans, off = [], 0
        for li, i in enumerate(idx):
            # tensor id of layer li of image 0 in the full set's numbering
            spans.append((40000 + s_idx * RESNET_IMAGES * per_img + li, off, ts.sizes[i]))
            off += ts.sizes[i]
        parts.append((O.params(ring, lx, c), s0, s1, spans))

    def step(m):
        for P, s0, s1, spans in parts:
            for tid, off, size in spans:
                if off >= m:
                    break
                e = min(off + size, m)
                O.relu(P, s0[off:e], s1[off:e], seed, tid, threads=threads)
        return 2 * m

    m0 = 1 << 15
    t0 = time.perf_counter()
    step(m0)
    per = (time.perf_counter() - t0) / (2 * m0)
    total_steps = max(1, args.steps + args.warmup)
    cap = min(p[1].size for p in parts)
    m = int(max(1 << 12, min(cap, 120.0 / (per * 2 * total_steps))))
    for _ in range(args.warmup):
        step(m)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(m)
    dt = time.perf_counter() - t0
    value = 2 * m * args.steps / dt
    total = RESNET_IMAGES * sum(W.RESNET18_224_LAYERS) * 2
    sample = (f"the oracle's ReLU on the first {m:,} elements of each ring's part of the set "
              f"per step ({2 * m:,} of {total:,} elements)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "elems/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+u32", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(images=RESNET_IMAGES, tensors=2 * RESNET_IMAGES
                                               * per_img, elems=f"{total:,}"),
                   "images": RESNET_IMAGES, "elements": total, "sample_per_step": 2 * m},
        "cpu_baseline": {"value": value, "unit": "elems/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "elems/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "parties3":
        parties3(args)              # spawns its own three processes; no CUDA in this one
        return
    import torch
    import torch.distributed as dist

    if args.serving_only:
        serving_only(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)          # before NCCL, so each rank binds its own GPU
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    try:
        if args.workload == "b1-pair":
            b1_pair(args, local, dev)
        elif args.workload == "fused":
            fused_main(args, world, rank, local, dev)
        else:
            headline(args, world, rank, local, dev)
    finally:
        if world > 1:
            dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the headline: the batched ResNet-18 ReLU set in both rings
# ---------------------------------------------------------------------------

def resnet18_items(ctx, dev, images, seed, tid_base=40000):
    """The ResNet-18 224x224 ReLU set of `images` images, shared on the device
    (Laplace(0, 2) reals; l = 64 with f = 16 and l = 32 with f = 12).  Returns
    the batch items (tensor id tid_base + index in the set), the
    (elements, l, lx) of each parameter group, the device buffers, and the
    tensor sizes in item order."""
    import torch
    from paper_2309_04909_gb300 import Params, workloads as W
    ts = W.resnet18_mixed_batch(images, seed=seed)
    items, parts, keep, sizes = [], [], [], []
    for ring, frac, prm in ((64, 16, Params(64, 24, 0)), (32, 12, Params(32, 14, 4))):
        idx = [i for i in range(len(ts.sizes)) if ts.ring_bits[i] == ring]
        allx = np.concatenate([np.rint(np.ldexp(ts.reals[i], frac)).astype(np.int64) for i in idx])
        for i in idx:
            ts.reals[i] = None
        s0, s1 = ctx.share(ring, torch.from_numpy(allx).to(dev), tensor_id=30 + ring)
        dt = torch.int64 if ring > 32 else torch.int32
        o0 = torch.empty(allx.size, dtype=dt, device=dev)
        o1 = torch.empty_like(o0)
        keep += [s0, s1, o0, o1]
        off = 0
        for i in idx:
            sl = slice(off, off + ts.sizes[i])
            items.append((prm, s0[sl], s1[sl], o0[sl], o1[sl], tid_base + i))
            sizes.append(ts.sizes[i])
            off += ts.sizes[i]
        parts.append((int(allx.size), ring, prm.lx))
        del allx
    return items, parts, keep, sizes


def batched_mul_ops(parts):
    from paper_2309_04909_gb300 import costmodel
    return sum(n * costmodel.mul_ops_per_element(lx, ring, relu=True) for n, ring, lx in parts)


def timed_over_ranks(step, steps, warmup, world, timer):
    """W untimed warm-up steps, then exactly `steps` timed steps bracketed by a
    barrier and a synchronisation on both sides; returns (own ms, max over
    ranks ms).  `timer` gives start()/stop() -> ms and sync() (CUDA events on
    the launching stream on the GPU)."""
    import torch.distributed as dist
    from paper_2309_04909_gb300.replicas import max_over_ranks
    for _ in range(max(3, warmup)):
        step()
    timer.sync()
    if world > 1:
        dist.barrier()
    timer.sync()
    timer.start()
    for _ in range(steps):
        step()
    own = timer.stop()
    if world > 1:
        dist.barrier()
    return own, max_over_ranks(own, device=timer.device)


class CudaTimer:
    """CUDA events on torch's current stream (the stream the library launches
    on); stop() synchronises."""

    def __init__(self, device):
        import torch
        self.device = device
        self._t = torch
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)

    def sync(self):
        self._t.cuda.synchronize()

    def start(self):
        self.a.record()

    def stop(self):
        self.b.record()
        self._t.cuda.synchronize()
        return self.a.elapsed_time(self.b)


def headline(args, world, rank, local, dev):
    import torch
    from paper_2309_04909_gb300 import Context, costmodel
    from paper_2309_04909_gb300.batch import DEFAULT_LAUNCH, ReluBatch, autotune
    from paper_2309_04909_gb300.replicas import rank_seed, shard_by_size

    ctx = Context(rank_seed(BASE_SEED, rank), device=local)
    # each rank its own batch of the same shape (weak scaling: replicas)
    items, parts, keep, sizes = resnet18_items(ctx, dev, args.images, seed=3 + rank)
    total = sum(p[0] for p in parts)
    torch.cuda.synchronize()
    best = (dict(DEFAULT_LAUNCH) if args.no_autotune
            else autotune(ctx, items, reps=1, use_cache=False))
    cfg = (best["tile_elems"], best["ctas_per_sm"], best["schedule"], best["elems_per_thread"],
           best["slot_unroll"])
    b = ReluBatch(ctx, items, *cfg)
    b.capture()
    launches_per_step = len(parts)          # one batched kernel per parameter group
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    own_ms, total_ms = timed_over_ranks(b.run, args.steps, args.warmup, world, CudaTimer(dev))
    ck = clocks.stop() if clocks else None
    assert b.status() == 0, "batched kernel reported a malformed tile"
    step_ms = own_ms / args.steps
    value = total * args.steps * world / (total_ms / 1e3)
    muls = batched_mul_ops(parts)
    peak = costmodel.int_mul_peak_ops()
    achieved = muls / (step_ms / 1e3)
    hbm = sum(n * costmodel.hbm_bytes_per_element_relu(ring) for n, ring, _ in parts)
    workload = WORKLOAD.format(images=args.images, tensors=len(items), elems=f"{total:,}")
    line = {
        "metric": METRIC, "value": value, "unit": "elems/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+u32",
        "data": "synthetic",
        "config": {"workload": workload, "images": args.images, "tensors": len(items),
                   "elements": total,
                   "groups": [{"ring_bits": r, "lx": lx, "key_off": 0 if r == 64 else 4,
                               "elements": n} for n, r, lx in parts],
                   "schedule": "grid" if best["schedule"] == 1 else "persistent",
                   "tile_elems": best["tile_elems"], "ctas_per_sm": best["ctas_per_sm"],
                   "elems_per_thread": best["elems_per_thread"],
                   "slot_unroll": best["slot_unroll"],
                   "parallelism": f"replicas x{world}",
                   "l2": f"working set {hbm / 1e9:.1f} GB per step > 129 MB L2; no flush"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T int32 multiply lane-ops/s", "frac": achieved / peak,
                     # DRAM bytes per step: ncu dram__bytes_read+write of both launches per
                     # element of a smaller set of the same mix, scaled to this step
                     "traffic": (TRAFFIC_PER_ELEM_BATCH * total
                                 if TRAFFIC_PER_ELEM_BATCH else None),
                     "kernel": "relu_batch_grid_kernel: the step's launches (l=64 lx=24, "
                               "l=32 lx=14), timed together" if best["schedule"] == 1 else
                               "relu_batch_kernel (persistent): the step's launches",
                     "kernel_ms": step_ms, "mul_ops_per_step": muls,
                     "peak_basis": "integer multiplier: 152 SM x 4 x 16-lane FMA-heavy pipe "
                                   "x 2070 MHz (maximum SM clock)",
                     "algorithmic_hbm_bytes_per_step": hbm,
                     "hbm_frac_of_measured": hbm / (step_ms / 1e3) / 6796.5e9},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck,
    }
    if world > 1:
        # strong scaling beside the weak replicas: the 1,088 tensors of ONE set
        # split over the ranks by size (each tensor whole on one rank)
        shard = shard_by_size(sizes, world)[rank]
        mine = [items[i] for i in shard]
        bs = ReluBatch(ctx, mine, *cfg)
        bs.capture()
        _, strong_ms = timed_over_ranks(bs.run, args.steps, args.warmup, world, CudaTimer(dev))
        line["strong_scaling"] = {
            "value": total * args.steps / (strong_ms / 1e3), "unit": "elems/s",
            "ms_per_step": strong_ms / args.steps,
            "split": "replicas.shard_by_size over the tensors of one set (largest first onto "
                     "the least loaded rank)",
            "tensors_on_rank0": len(shard)}
    if not args.no_extras:
        line["e2e"] = headline_e2e(ctx, items, cfg, min(args.steps, 20), world, dev)
    if rank == 0 and world == 1 and not args.no_extras:
        headline_extras(args, line, ctx, items, parts, cfg, step_ms, local, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    del b
    ctx.close()


_LINK = {}


def host_link_gbps(nbytes: int = 256 << 20, reps: int = 4) -> dict:
    """This machine's host link, measured once per process with copy engines:
    H2D alone, D2H alone and both at once (pinned buffers, CUDA events on
    two streams).  The e2e rooflines divide by the bidirectional figure; it
    differs between boxes of the pool (316-340 GB/s on most, about 130 on
    one), so a fixed constant would misstate the fraction."""
    import torch
    if _LINK:
        return _LINK
    n = nbytes // 4
    h_in = torch.ones(n, dtype=torch.int32).pin_memory()
    h_out = torch.empty(n, dtype=torch.int32).pin_memory()
    d_in = torch.empty(n, dtype=torch.int32, device="cuda")
    d_out = torch.ones(n, dtype=torch.int32, device="cuda")
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(up: bool, down: bool) -> float:
        for _ in range(2):
            if up:
                with torch.cuda.stream(s_up):
                    d_in.copy_(h_in, non_blocking=True)
            if down:
                with torch.cuda.stream(s_down):
                    h_out.copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        ends = []
        for st, on in ((s_up, up), (s_down, down)):
            if not on:
                continue
            st.wait_event(start)
            with torch.cuda.stream(st):
                for _ in range(reps):
                    if st is s_up:
                        d_in.copy_(h_in, non_blocking=True)
                    else:
                        h_out.copy_(d_out, non_blocking=True)
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                ends.append(e)
        torch.cuda.synchronize()
        ms = max(start.elapsed_time(e) for e in ends)
        return (int(up) + int(down)) * reps * nbytes / (ms * 1e-3) / 1e9

    _LINK.update({"h2d_GBps": timed(True, False), "d2h_GBps": timed(False, True),
                  "both_GBps": timed(True, True),
                  "how": "copy engines, pinned 256 MB buffers, H2D and D2H on two streams at "
                         "once for both_GBps; measured on this box before the e2e run"})
    return _LINK


def headline_e2e(ctx, items, cfg, steps, world, dev):
    """The headline step through the host-buffer entry point
    (bc_relu_batch_host): the input shares in page-locked host memory, the
    output shares written back to page-locked host memory, every step; the
    batched kernel reads and writes them across the host link.  Checked equal
    to the device-resident run's outputs."""
    import torch
    from paper_2309_04909_gb300.replicas import max_over_ranks
    # one page-locked array per ring and share (the batch's activations of a
    # ring live in one buffer), sliced per tensor like the device arrays
    host = []
    h2d = d2h = 0
    rings = sorted({it[0].ring_bits for it in items})
    for ring in rings:
        its = [it for it in items if it[0].ring_bits == ring]
        n = sum(it[1].numel() for it in its)
        dt = its[0][1].dtype
        arrs = [torch.empty(n, dtype=dt).pin_memory() for _ in range(4)]
        off = 0
        for prm, s0, s1, o0, o1, tid in its:
            m = s0.numel()
            sl = [a[off:off + m] for a in arrs]
            sl[0].copy_(s0)
            sl[1].copy_(s1)
            host.append((prm, sl[0], sl[1], sl[2], sl[3], tid))
            off += m
            h2d += 2 * m * s0.element_size()
            d2h += 2 * m * o0.element_size()
    ref = {it[5]: it for it in items}
    # the descriptors name the buffers (addresses and sizes), built once like a
    # C caller's bc_tensor_desc array; every step plans, runs and synchronises
    descs, count = ctx.batch_descs(host)
    run = lambda: ctx.relu_batch_host_descs(descs, count, *cfg)
    for _ in range(3):
        run()
    equal = all(torch.equal(h[3], ref[h[5]][3].cpu()) and torch.equal(h[4], ref[h[5]][4].cpu())
                for h in host)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        run()
    dt = max_over_ranks(time.perf_counter() - t0, device=dev)
    total = sum(it[1].numel() for it in items)
    meas = host_link_gbps()
    link = meas["both_GBps"]
    value = total * steps * world / dt
    return {"value": value, "unit": "elems/s", "h2d_bytes_per_step": h2d * world,
            "d2h_bytes_per_step": d2h * world, "steps": steps, "equal_to_device_run": equal,
            "api": "bc_relu_batch_host on a prepared descriptor array: pinned host input and "
                   "output shares (one page-locked array per ring and share, sliced per "
                   "tensor); the batched kernel loads and stores them across the host link; "
                   "plan + run + synchronise every step",
            "link_roofline": {"bytes_per_step": h2d + d2h, "link_GBps": link,
                              "bound_elems_per_s": world * link * 1e9 * total / (h2d + d2h),
                              "frac": value / (world * link * 1e9 * total / (h2d + d2h)),
                              "link": meas}}


def oracle_relu_sample(ctx, items, per_ring, threads):
    """The oracle's ReLU on the first `per_ring` elements of each ring's part
    of the batch (whole tensors in order, the last one cut), on the device's
    own input shares copied to the host, with `threads` OpenMP threads.
    Returns (elements, seconds of oracle time)."""
    import oracle as O
    done = {}
    elems, secs = 0, 0.0
    for prm, s0, s1, o0, o1, tid in items:
        left = per_ring - done.get(prm.ring_bits, 0)
        if left <= 0:
            continue
        m = min(left, s0.numel())
        a0 = s0[:m].cpu().numpy().view(np.uint64 if prm.ring_bits > 32 else np.uint32)
        a1 = s1[:m].cpu().numpy().view(np.uint64 if prm.ring_bits > 32 else np.uint32)
        P = O.params(prm.ring_bits, prm.lx, prm.key_off)
        t0 = time.perf_counter()
        O.relu(P, a0, a1, ctx.seed, tid, threads=threads)
        secs += time.perf_counter() - t0
        done[prm.ring_bits] = done.get(prm.ring_bits, 0) + m
        elems += m
    return elems, secs


def headline_extras(args, line, ctx, items, parts, cfg, step_ms, local, dev):
    """Single-GPU extras of the headline (each recorded under its key; a
    failing extra records its error and the line still prints): the measured
    multiplier rates, the CPU oracle on a sample of the same set, the
    per-tensor launches it replaces, and then the fused linear-layer step and
    the other workloads."""
    import torch
    from paper_2309_04909_gb300 import costmodel

    def extra(key, fn, into=None):
        try:
            (into if into is not None else line)[key] = fn()
        except Exception as exc:   # noqa: BLE001 - recorded, the headline stands
            (into if into is not None else line)[key] = {"error": f"{type(exc).__name__}: {exc}"}
            try:
                torch.cuda.synchronize()
            except Exception:      # noqa: BLE001 - a sticky CUDA error is already recorded
                pass

    def measured_rates():
        # the multiplier's rates measured by our own microbenchmark (after the
        # timed region): the time the step's algorithmic products need at
        # those rates, against the step's time
        from paper_2309_04909_gb300 import measure_int_peaks
        mp = measure_int_peaks(local)
        w = lo = hi = 0
        for n, ring, lx in parts:
            a, b, c = costmodel.mul_counts_split(lx, ring, relu=True)
            w, lo, hi = w + n * a, lo + n * b, hi + n * c
        bound_ms = (w / mp["imad_wide_per_s"] + lo / mp["imad_per_s"]
                    + hi / mp["imad_hi_per_s"]) * 1e3
        return {"widening_products": w, "low_products": lo, "high_products": hi,
                "imad_wide_per_s": mp["imad_wide_per_s"], "imad_per_s": mp["imad_per_s"],
                "imad_hi_per_s": mp["imad_hi_per_s"], "alu_per_s": mp["alu_per_s"],
                "sm_mhz": mp["sm_mhz"], "bound_ms": bound_ms, "frac": bound_ms / step_ms,
                "basis": "widening products timed as Philox-4x32 rounds, low products as "
                         "32-bit multiply-adds, high products as hi32(x k) chains; "
                         "full-occupancy microbenchmark on this GPU"}

    def cpu_baseline():
        import oracle as O
        total = sum(p[0] for p in parts)
        cores = O.max_threads()
        per = 1 << 23
        m, dt = oracle_relu_sample(ctx, items, per, cores)
        m1, dt1 = oracle_relu_sample(ctx, items, 1 << 18, 1)
        return {"value": m / dt, "unit": "elems/s", "cores": cores, "kind": "oracle",
                "sample": f"the oracle's ReLU on the first {per:,} elements of each ring's "
                          f"part of the set ({m:,} elements, input shares from the device), "
                          f"{dt:.1f} s; full set extrapolated to {total * dt / m:.0f} s",
                "full_set_seconds_extrapolated": total * dt / m,
                "single_thread": {"value": m1 / dt1, "sample_elems": m1, "seconds": dt1}}

    def plain():
        # one launch per tensor (the single-tensor kernel), replayed from a
        # CUDA graph, against the batched graph; identical outputs
        q = [(torch.empty_like(it[3]), torch.empty_like(it[4])) for it in items]

        def run_plain():
            for it, (a, b) in zip(items, q):
                ctx.relu(it[0], it[1], it[2], it[5], out=(a, b))

        run_plain()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run_plain()
        plain_ms = median_ms(g.replay)
        same = all(torch.equal(it[3], a) and torch.equal(it[4], b) for it, (a, b) in zip(items, q))
        return {"plain_graph_ms": plain_ms, "batched_graph_ms": step_ms,
                "speedup_vs_plain_graph": plain_ms / step_ms, "plain_launches": len(items),
                "batched_launches": len(parts), "identical_to_plain": bool(same),
                "timing": "plain: median of 20 graph replays, CUDA events per run; batched: the "
                          "headline's timed steps"}

    extra("measured_rates", measured_rates, into=line["roofline"])
    extra("cpu_baseline", cpu_baseline)
    extra("batched_vs_plain_resnet18", plain)
    # the fused linear-layer step and the other workloads
    try:
        fl, state = fused_step(args, 1, 0, local, dev, steps=args.fused_steps)
        line["fused_step_l64_2p22"] = fl
        run_extras(args, line, *state)
        state[0].close()
    except Exception as exc:   # noqa: BLE001 - recorded, the headline stands
        line["fused_step_l64_2p22"] = {"error": f"{type(exc).__name__}: {exc}"}


# ---------------------------------------------------------------------------
# the fused step of a linear layer (product -> truncations -> ReLU)
# ---------------------------------------------------------------------------

def fused_main(args, world, rank, local, dev):
    """`--workload fused`: the fused step alone as the line (for profiling),
    or its chain / party-separated / RSS variants with --step."""
    line, state = fused_step(args, world, rank, local, dev, steps=args.steps)
    if line is None:
        return
    if not args.no_extras:
        ctx, prm, x0, x1, y0, y1 = state[:6]
        n = state[9]
        line["e2e"] = e2e_all_ranks(ctx, prm, x0, x1, y0, y1, n, min(args.steps, 100), world,
                                    dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    state[0].close()


def fused_step(args, world, rank, local, dev, steps):
    """Times `steps` fused steps (one kernel each) at N = args.n; returns the
    line of that step and the state the extras read."""
    import torch
    from paper_2309_04909_gb300 import Context, Params, costmodel
    from paper_2309_04909_gb300.replicas import rank_seed

    n = args.n
    xi, yi = workload_inputs(n, seed=SEED + rank)   # each rank its own batch (replicas)
    ctx = Context(rank_seed(BASE_SEED, rank), device=local)
    x0, x1 = ctx.share(RING, torch.from_numpy(xi).to(dev), tensor_id=1)
    y0, y1 = ctx.share(RING, torch.from_numpy(yi).to(dev), tensor_id=2)
    prm = Params(RING, LX, KEY_OFF)
    buf = ctx.linear_relu_buffers(RING, K_TRUNC, n)
    # the step's outputs: the ReLU of the SecureML-truncated product and the
    # deterministic truncation; product and truncated shares stay in registers
    work = {nm: buf[nm] for nm in ("det0", "det1", "relu0", "relu1")}
    torch.cuda.synchronize()

    def step():
        ctx.linear_relu(RING, K_TRUNC, prm, x0, x1, y0, y1, tensor_id=3, work=work)

    if args.workload == "fused" and args.step == "chain":
        chain_only(args, ctx, prm, x0, x1, y0, y1, buf, n, world, dev)
        ctx.close()
        return None, None
    if args.workload == "fused" and args.step in ("parties", "rss"):
        variant_only(args, ctx, prm, x0, x1, y0, y1, buf, n, world, dev)
        ctx.close()
        return None, None

    # the step is exactly one launch of the fused kernel, so the start/end
    # events on its stream time the kernel back to back: no per-step events,
    # which would add their own gaps between launches
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    own_ms, total_ms = timed_over_ranks(step, steps, args.warmup, world, CudaTimer(dev))
    ck = clocks.stop() if clocks else None
    kern_ms = own_ms / steps        # average launch duration of the fused kernel
    value = n * steps * world / (total_ms / 1e3)
    ops = costmodel.linear_relu_int_ops_per_element(LX, RING)
    muls = costmodel.linear_relu_mul_ops_per_element(LX, RING)
    peak = costmodel.int_mul_peak_ops()
    achieved = muls * n / (kern_ms / 1e3)
    issue_frac = ops * n / (kern_ms / 1e3) / costmodel.int_issue_peak_ops()
    line = {
        "metric": METRIC, "value": value, "unit": "elems/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": FUSED_WORKLOAD, "n": n, "ring_bits": RING, "frac_bits": FRAC,
                   "trunc_bits": K_TRUNC, "lx": LX, "key_off": KEY_OFF, "p": 16777259,
                   "parallelism": f"replicas x{world}",
                   "l2": "working set 268 MB per step > 129 MB L2; no flush"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T int32 multiply lane-ops/s", "frac": achieved / peak,
                     # DRAM bytes per launch: ncu dram__bytes_read+write of this kernel
                     # per element, scaled to this launch's n
                     "traffic": TRAFFIC_PER_ELEM * n if TRAFFIC_PER_ELEM else None,
                     "kernel": "linear_relu_kernel<uint64_t,24,SHORT>",
                     "mul_ops_per_element": muls, "kernel_ms": kern_ms,
                     "peak_basis": "integer multiplier: 152 SM x 4 x 16-lane FMA-heavy pipe "
                                   "x 2070 MHz (maximum SM clock)",
                     "int_ops_per_element": ops,
                     "issue_frac": issue_frac,
                     "hbm_bytes_per_element": costmodel.hbm_bytes_per_element_linear_relu(RING)},
        "gpu_launches": steps,
        "clocks": ck,
    }
    if rank == 0 and not args.no_extras:
        from paper_2309_04909_gb300 import measure_int_peaks
        mp = measure_int_peaks(local)
        w, lo, hi = costmodel.mul_counts_split(LX, RING, relu=True, product=True)
        bound_ms = n * (w / mp["imad_wide_per_s"] + lo / mp["imad_per_s"]
                        + hi / mp["imad_hi_per_s"]) * 1e3
        line["roofline"]["measured_rates"] = {
            "widening_products_per_element": w, "low_products_per_element": lo,
            "high_products_per_element": hi,
            "imad_wide_per_s": mp["imad_wide_per_s"], "imad_per_s": mp["imad_per_s"],
            "imad_hi_per_s": mp["imad_hi_per_s"], "alu_per_s": mp["alu_per_s"],
            "sm_mhz": mp["sm_mhz"], "bound_ms": bound_ms, "frac": bound_ms / kern_ms}
    state = (ctx, prm, x0, x1, y0, y1, xi, yi, buf, n, kern_ms, dev)
    return line, state


def run_extras(args, line, ctx, prm, x0, x1, y0, y1, xi, yi, buf, n, kern_ms, dev):
    """The single-GPU extras, each recorded under its key.  An extra that
    fails records its error instead, so the headline line is always printed."""
    import torch

    def extra(key, fn, into=None):
        try:
            (into if into is not None else line)[key] = fn()
        except Exception as exc:   # noqa: BLE001 - recorded, the headline stands
            (into if into is not None else line)[key] = {"error": f"{type(exc).__name__}: {exc}"}
            try:
                torch.cuda.synchronize()
            except Exception:      # noqa: BLE001 - a sticky CUDA error is already recorded
                pass

    def cpu_baseline():
        rate, m2, dt = cpu_rate(args.cpu_seconds, xi, yi, _threads())
        rate1, m1, dt1 = cpu_rate(max(2.0, args.cpu_seconds / 5), xi, yi, 1)
        return {"value": rate, "unit": "elems/s", "cores": _threads(), "kind": "oracle",
                "sample": f"first {m2} elements of the workload, full step "
                          f"(share, product, both truncations, ReLU), {dt:.1f} s",
                "single_thread": {"value": rate1, "sample_elems": m1, "seconds": dt1}}

    # the fused linear-layer step's own extras go under its key
    fl = line.setdefault("fused_step_l64_2p22", {})
    extra("e2e", lambda: e2e_all_ranks(ctx, prm, x0, x1, y0, y1, n, 100, 1, dev), into=fl)
    # every intermediate of the step, for the extras that read them
    ctx.linear_relu(RING, K_TRUNC, prm, x0, x1, y0, y1, tensor_id=3, work=buf)
    extra("unfused_chain", lambda: chain_bench(ctx, prm, x0, x1, y0, y1, buf, n, kern_ms),
          into=fl)
    if "error" not in fl.get("e2e", {"error": 1}):
        extra("paths", lambda: e2e_paths(ctx, prm, x0, x1, y0, y1, n, 30, buf), into=fl["e2e"])
    extra("trunc_failures", lambda: trunc_failures(ctx, xi, yi, x0, x1, y0, y1, buf, dev),
          into=fl)
    extra("cpu_baseline", cpu_baseline, into=fl)
    relu_ms = fl["unfused_chain"].get("relu_ms", kern_ms)
    extra("party_separated", lambda: parties_bench(ctx, prm, buf, n, relu_ms), into=fl)
    extra("rss_relu", lambda: rss_bench(ctx, prm, buf, n), into=fl)
    extra("bicoptor1_vs_2", lambda: b1_bench(ctx, x0, x1, n))
    # the other workloads
    extra("hbm_kernels_isolated", lambda: hbm_isolated(ctx, dev))
    extra("linear_layer_truncation", lambda: linear_trunc_table(ctx, dev))
    extra("cpu_baseline_batched_configs", lambda: cpu_configs(_threads()))
    extra("drelu_l32_uniform", lambda: uniform_l32_drelu_check(ctx, dev))
    extra("size_sweep_l64", lambda: size_sweep(ctx, dev))
    if "error" not in line.get("size_sweep_l64", {"error": 1}):
        extra("network_projection", lambda: network_projection(line["size_sweep_l64"]))
    extra("batched_vs_plain", lambda: vgg16_batched_vs_plain(ctx, dev))
    bvp = line["batched_vs_plain"]
    if "batched_elems_per_s" in bvp:
        extra("serving", lambda: serving_bench(ctx, dev, bvp["batched_elems_per_s"],
                                               args.serve_seconds, args.serve_load_seconds,
                                               bvp))


def _threads():
    import oracle as O
    return O.max_threads()


def chain_bench(ctx, prm, x0, x1, y0, y1, buf, n, fused_ms, steps=20, warmup=3):
    """The step as four separate launches (Beaver product, the two
    truncations, ReLU) through HBM, each kernel timed with CUDA events, and
    checked bit for bit against the fused kernel's outputs."""
    import torch
    hbm_peak = 6793.4   # GB/s, measured STREAM-style copy on the GB300s
    q = {nm: torch.empty_like(t) for nm, t in buf.items()}

    def run(ev=None):
        rec = (lambda j: ev[j].record()) if ev else (lambda j: None)
        rec(0)
        ctx.mul_beaver(RING, x0, x1, y0, y1, 3, out=(q["prod0"], q["prod1"]))
        rec(1)
        ctx.trunc_prob(RING, K_TRUNC, q["prod0"], q["prod1"], out=(q["trc0"], q["trc1"]))
        rec(2)
        ctx.trunc_det(RING, K_TRUNC, 0, q["prod0"], q["prod1"], out=(q["det0"], q["det1"]))
        rec(3)
        ctx.relu(prm, q["trc0"], q["trc1"], 4, out=(q["relu0"], q["relu1"]))
        rec(4)

    for _ in range(warmup):
        run()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    for ev in evs:
        run(ev)
    torch.cuda.synchronize()
    ms = [sum(ev[j].elapsed_time(ev[j + 1]) for ev in evs) / len(evs) for j in range(4)]
    same = all(torch.equal(q[nm], buf[nm]) for nm in buf)

    def hbm(t, bytes_per_elem):
        gbs = bytes_per_elem * n / (t / 1e3) / 1e9
        return {"ms": t, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm_peak,
                "bytes_per_element": bytes_per_elem}
    return {"ms": sum(ms), "fused_ms": fused_ms,
            "speedup_of_fusion": sum(ms) / fused_ms if fused_ms else None,
            "relu_ms": ms[3], "equal_to_fused": same if fused_ms else None,
            "hbm_kernels": {"mul_beaver": hbm(ms[0], 48), "trunc_prob": hbm(ms[1], 32),
                            "trunc_det": hbm(ms[2], 32)}}


def hbm_isolated(ctx, dev, log2n=25, iters=20, warmup=3):
    """Each HBM-bound kernel of the C-ABI alone, at 2^25 elements: every l = 64
    array is 256 MiB, twice the 129 MB L2, so every launch reads its inputs
    from HBM.  Each kernel is timed with CUDA events around `iters`
    back-to-back launches on the context's stream."""
    import torch
    from paper_2309_04909_gb300 import prime_above
    hbm_peak = 6793.4   # GB/s, measured STREAM-style copy on the GB300s
    n = 1 << log2n
    g = torch.Generator(device=dev).manual_seed(0x4B4D)
    lo, hi = -(1 << 63), (1 << 63) - 1

    def u64():
        return torch.randint(lo, hi, (n,), dtype=torch.int64, device=dev, generator=g)

    x0, x1, y0, y1 = u64(), u64(), u64(), u64()
    xf = torch.randint(-(1 << 40), 1 << 40, (n,), dtype=torch.int64, device=dev, generator=g)
    m0 = torch.randint(0, 1 << 24, (n,), dtype=torch.int32, device=dev, generator=g)
    m1 = torch.randint(0, 1 << 24, (n,), dtype=torch.int32, device=dev, generator=g)
    o0, o1 = torch.empty_like(x0), torch.empty_like(x0)
    p24 = prime_above(24)
    kernels = {
        # name: (call, algorithmic bytes per element)
        "share": (lambda: ctx.share(RING, xf, 7), 24),
        "reconstruct": (lambda: ctx.reconstruct(RING, x0, x1), 24),
        "trunc_prob": (lambda: ctx.trunc_prob(RING, K_TRUNC, x0, x1, out=(o0, o1)), 32),
        "trunc_det": (lambda: ctx.trunc_det(RING, K_TRUNC, 0, x0, x1, out=(o0, o1)), 32),
        "mod_switch_lx24": (lambda: ctx.mod_switch(24, p24, m0, m1), 16),
        "mul_beaver": (lambda: ctx.mul_beaver(RING, x0, x1, y0, y1, 8, out=(o0, o1)), 48),
    }
    out = {"n": n, "iters": iters, "hbm_peak_GB/s": hbm_peak, "l2": "inputs > L2 (no flush)"}
    for name, (call, bpe) in kernels.items():
        for _ in range(warmup):
            call()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        for _ in range(iters):
            call()
        e.record()
        torch.cuda.synchronize()
        us = s.elapsed_time(e) * 1e3 / iters
        gbs = bpe * n / (us / 1e6) / 1e9
        out[name] = {"us": us, "bytes_per_element": bpe, "GB/s": gbs,
                     "frac_of_measured_hbm": gbs / hbm_peak}
    return out


def chain_only(args, ctx, prm, x0, x1, y0, y1, buf, n, world, dev):
    """`--step chain`: the step as four launches through HBM (the standalone
    kernels of the C-ABI), each timed with CUDA events on its stream; the
    ReLU kernel's roofline is reported."""
    import torch
    from paper_2309_04909_gb300 import costmodel
    from paper_2309_04909_gb300.replicas import max_over_ranks
    r = chain_bench(ctx, prm, x0, x1, y0, y1, buf, n, None, steps=args.steps,
                    warmup=max(3, args.warmup))
    total = max_over_ranks(r["ms"], device=dev)
    muls = costmodel.mul_ops_per_element(LX, RING, relu=True)
    peak = costmodel.int_mul_peak_ops()
    achieved = muls * n / (r["relu_ms"] / 1e3)
    line = {"metric": METRIC, "value": n * world / (total / 1e3), "unit": "elems/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": FUSED_WORKLOAD + " (four launches)", "n": n},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                         "unit": "T int32 multiply lane-ops/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "relu_kernel<uint64_t,24,SHORT,ReLU>",
                         "mul_ops_per_element": muls, "kernel_ms": r["relu_ms"]},
            "gpu_launches": 4 * args.steps, "chain": r}
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)


def variant_only(args, ctx, prm, x0, x1, y0, y1, buf, n, world, dev):
    """`--step parties` / `--step rss`: the ReLU of the step's truncated
    product by the party-separated launches (messages in device buffers) or
    by the RSS protocol, timed as the step (for profiling those paths)."""
    import torch
    from paper_2309_04909_gb300.replicas import max_over_ranks
    ctx.linear_relu(RING, K_TRUNC, prm, x0, x1, y0, y1, tensor_id=3, work=buf)
    if args.step == "parties":
        msgs = ctx.party_buffers(prm, n)
        out = (torch.empty_like(buf["relu0"]), torch.empty_like(buf["relu1"]))
        run = lambda: ctx.relu_parties(prm, buf["trc0"], buf["trc1"], 4, out=out, msgs=msgs)
        launches = 3
    else:
        z = torch.zeros_like(buf["trc0"])
        ys = tuple(torch.empty_like(buf["trc0"]) for _ in range(3))
        run = lambda: ctx.rss_relu(prm, buf["trc0"], z, buf["trc1"], 4, out=ys)
        launches = 1
    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
    line = {"metric": METRIC, "value": n * world / (ms / 1e3), "unit": "elems/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"ReLU of the step's truncated product, {args.step} path",
                       "n": n},
            "gpu_launches": launches * args.steps}
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)


def _host_step_inputs(x0, x1, y0, y1, n):
    import torch
    hx = [t.cpu().pin_memory() for t in (x0, x1, y0, y1)]
    out = {k: torch.empty(n, dtype=torch.int64).pin_memory()
           for k in ("relu0", "relu1", "det0", "det1")}
    return hx, out


def e2e_all_ranks(ctx, prm, x0, x1, y0, y1, n, steps, world, dev):
    """The step through the host-buffer entry point (the call a user with
    host data makes): pinned host inputs and outputs, host<->device transfers
    inside the timed region, default path.  Every rank runs its own batch
    between barriers; the time is the max over ranks."""
    import torch
    import torch.distributed as dist
    from paper_2309_04909_gb300.replicas import max_over_ranks
    hx, out = _host_step_inputs(x0, x1, y0, y1, n)
    for _ in range(5):          # first touches of the fresh pinned pages stay out of the timing
        ctx.linear_relu_host(RING, K_TRUNC, prm, *hx, tensor_id=3, out=out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.linear_relu_host(RING, K_TRUNC, prm, *hx, tensor_id=3, out=out)
    dt = max_over_ranks(time.perf_counter() - t0, device=dev)
    value = n * steps * world / dt
    meas = host_link_gbps()
    link = meas["both_GBps"]
    return {"value": value, "unit": "elems/s", "h2d_bytes_per_step": 4 * 8 * n * world,
            "d2h_bytes_per_step": 4 * 8 * n * world, "steps": steps,
            "api": "bc_linear_relu_host, pinned host buffers, default path (direct: the fused "
                   "kernel loads and stores them across the host link)",
            "link_roofline": {"bytes_per_element": 64, "link_GBps": link,
                              "bound_elems_per_s": world * link * 1e9 / 64,
                              "frac": value / (world * link * 1e9 / 64), "link": meas}}


def e2e_paths(ctx, prm, x0, x1, y0, y1, n, steps, buf):
    """Both host-buffer paths on one GPU: direct (the fused kernel loads and
    stores the pinned buffers across the host link) and staged (chunks copied
    through device buffers on four streams, best chunk of three), each
    checked against the device step's outputs."""
    import torch
    hx, out = _host_step_inputs(x0, x1, y0, y1, n)
    names = tuple(out)

    def timed(reps):
        ctx.linear_relu_host(RING, K_TRUNC, prm, *hx, tensor_id=3, out=out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.linear_relu_host(RING, K_TRUNC, prm, *hx, tensor_id=3, out=out)
        return n * reps / (time.perf_counter() - t0)

    def same():
        return all(torch.equal(out[k], buf[k].cpu()) for k in names)

    paths = {}
    ctx.set_host_path(ctx.HOST_STAGED)
    best = None
    for chunk_log2 in (18, 19, 20):
        ctx.reserve(1 << chunk_log2)
        r = timed(5)
        if best is None or r > best[1]:
            best = (chunk_log2, r)
    ctx.reserve(1 << best[0])
    paths["staged"] = {"elems_per_s": timed(steps), "chunk": 1 << best[0], "equal": same()}
    ctx.set_host_path(ctx.HOST_DIRECT)
    paths["direct"] = {"elems_per_s": timed(steps), "equal": same()}
    ctx.set_host_path(ctx.HOST_AUTO)
    return paths


def trunc_failures(ctx, xi, yi, x0, x1, y0, y1, buf, dev):
    """Probabilistic vs deterministic truncation failures against the
    plaintext, with the closed form sum |x| / 2^l, on the product and on a
    stress sweep of large-magnitude inputs."""
    import torch
    from paper_2309_04909_gb300 import workloads as W
    out = {}
    prod = torch.from_numpy(xi * yi).to(dev)        # |x y| < 2^63 for these inputs
    pf = ctx.count_trunc_failures(RING, K_TRUNC, prod, buf["trc0"], buf["trc1"])
    df = ctx.count_trunc_failures(RING - K_TRUNC, K_TRUNC, prod, buf["det0"], buf["det1"])
    expect = float(np.abs(xi.astype(np.float64) * yi.astype(np.float64)).sum() / 2.0**64)
    out["product"] = {"prob": pf, "det": df, "prob_expected": expect}
    sweep = {}
    n = 1 << 22
    for bits in (48, 56, 60, 62):
        x = W.magnitude_bounded_ints(n, bits, seed=bits)
        xg = torch.from_numpy(x).to(dev)
        s0, s1 = ctx.share(RING, xg, tensor_id=7000 + bits)
        p0, p1 = ctx.trunc_prob(RING, K_TRUNC, s0, s1)
        d0, d1 = ctx.trunc_det(RING, K_TRUNC, 0, s0, s1)
        sweep[str(bits)] = {
            "prob": ctx.count_trunc_failures(RING, K_TRUNC, xg, p0, p1),
            "det": ctx.count_trunc_failures(RING - K_TRUNC, K_TRUNC, xg, d0, d1),
            "prob_expected": float(np.abs(x.astype(np.float64)).sum() / 2.0**64)}
    out["stress_sweep_mag_bits"] = sweep
    return out


def batched_frac(parts, ms):
    """Fraction of the integer-multiplier roofline reached by a batched ReLU
    run: parts = (elements, l, lx) of each parameter class."""
    from paper_2309_04909_gb300 import costmodel
    ops = sum(n * costmodel.mul_ops_per_element(lx, ring, relu=True) for n, ring, lx in parts)
    return ops / (ms / 1e3) / costmodel.int_mul_peak_ops()


def b_persist_ms(ctx, items):
    """Best persistent-schedule time over the autotuner's tile candidates."""
    from paper_2309_04909_gb300.batch import TILE_CANDIDATES, ReluBatch, time_ms
    return min(time_ms(ReluBatch(ctx, items, t, c, 0).run, reps=3, warmup=1)
               for t in TILE_CANDIDATES for c in (0, 2))


def median_ms(fn, reps=20, warmup=3):
    """Median over `reps` runs of fn, each bracketed by its own CUDA events on
    the current stream.  The batched sets are larger than L2, so runs need no
    flush between them."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for st, en in evs:
        st.record()
        fn()
        en.record()
    torch.cuda.synchronize()
    return statistics.median(st.elapsed_time(en) for st, en in evs)


def vgg16_batched_vs_plain(ctx, dev, batch=128):
    """The 13 ReLU tensors of a VGG-16 on 32x32 inputs for
    `batch` images (1,664 tensors, 35,389,440 elements at batch 128), l = 64,
    f = 16, per-layer sigma in [0.5, 8].  Plain = one launch per tensor
    (eager, and replayed from a CUDA graph); batched = one persistent launch
    over the tile queue (autotuned tile / CTAs per SM), eager and graph."""
    import torch
    from paper_2309_04909_gb300 import Params, workloads as W
    from paper_2309_04909_gb300.batch import ReluBatch, autotune
    ts = W.vgg16_batch(batch, seed=2)
    allx = np.concatenate([np.rint(np.ldexp(r, 16)).astype(np.int64) for r in ts.reals])
    total = allx.size
    s0, s1 = ctx.share(64, torch.from_numpy(allx).to(dev), tensor_id=11)
    o0 = torch.empty(total, dtype=torch.int64, device=dev)
    o1 = torch.empty(total, dtype=torch.int64, device=dev)
    q0 = torch.empty_like(o0)
    q1 = torch.empty_like(o1)
    prm = Params(64, 24, 0)
    items, plain_items, off = [], [], 0
    for t, sz in enumerate(ts.sizes):
        sl = slice(off, off + sz)
        items.append((prm, s0[sl], s1[sl], o0[sl], o1[sl], 20000 + t))
        plain_items.append((prm, s0[sl], s1[sl], q0[sl], q1[sl], 20000 + t))
        off += sz

    def plain():
        for it in plain_items:
            ctx.relu(it[0], it[1], it[2], it[5], out=(it[3], it[4]))

    plain_ms = median_ms(plain)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        plain()
    plain_graph_ms = median_ms(g.replay)
    best = autotune(ctx, items, reps=2, use_cache=False)
    b = ReluBatch(ctx, items, best["tile_elems"], best["ctas_per_sm"], best["schedule"],
                  best["elems_per_thread"], best["slot_unroll"])
    batched_ms = median_ms(b.run)
    b.capture()
    batched_graph_ms = median_ms(b.run)
    identical = bool(torch.equal(o0, q0) and torch.equal(o1, q1))
    return {"workload": f"VGG-16 32x32 ReLU set, batch {batch}: {len(ts.sizes)} tensors, "
                        f"{total} elements, l=64 f=16 lx=24",
            "plain_eager_ms": plain_ms, "plain_graph_ms": plain_graph_ms,
            "batched_ms": batched_ms, "batched_graph_ms": batched_graph_ms,
            "speedup_vs_plain_eager": plain_ms / batched_graph_ms,
            "speedup_vs_plain_graph": plain_graph_ms / batched_graph_ms,
            "batched_elems_per_s": total / (batched_graph_ms / 1e3),
            "batched_roofline_frac": batched_frac([(total, 64, 24)], batched_graph_ms),
            "schedule": "grid" if best["schedule"] == 1 else "persistent",
            "tile_elems": best["tile_elems"], "ctas_per_sm": best["ctas_per_sm"],
            "elems_per_thread": best["elems_per_thread"], "slot_unroll": best["slot_unroll"],
            "persistent_best_ms": b_persist_ms(ctx, items),
            "timing": "median of 20 runs, CUDA events per run, after 3 warm-up runs",
            "status": b.status(), "identical_to_plain": identical}


def linear_trunc_table(ctx, dev, n=1 << 22):
    """Sec. 4 on synthetic products: x, y ~ N(0, 4^2) with f fractional bits
    in Z_{2^64} (5 integer bits), their product truncated by f:
      mult-then-trc, ABY3, random r     (e1 expected: sum |x y| / 2^64)
      mult-then-trc, ABY3, r = 2^f fixed (the shortcut that hides e1)
      mult-then-trc, SecureML
      trc-then-mult (Alg. linear)        (inputs truncated by f/2 first)
    Failures counted against floor(x y / 2^f) (more than one away)."""
    import torch
    from paper_2309_04909_gb300 import workloads as W
    out = {}
    for f in (13, 20, 26):
        X = W.gaussian_reals(n, 4.0, seed=40 + f, stream=0)
        Y = W.gaussian_reals(n, 4.0, seed=40 + f, stream=1)
        xi = np.rint(np.ldexp(X, f)).astype(np.int64)
        yi = np.rint(np.ldexp(Y, f)).astype(np.int64)
        prod = xi * yi                      # |x y| < 2^62 for these inputs: exact in int64
        x0, x1 = ctx.share(64, torch.from_numpy(xi).to(dev), tensor_id=500 + f)
        y0, y1 = ctx.share(64, torch.from_numpy(yi).to(dev), tensor_id=600 + f)
        p0, p1 = ctx.mul_beaver(64, x0, x1, y0, y1, tensor_id=700 + f)
        pg = torch.from_numpy(prod).to(dev)
        row = {"expected_e1_random_r": float(np.abs(prod.astype(np.float64)).sum() / 2.0 ** 64)}
        a0, a1 = ctx.trunc_aby3(64, f, p0, p1, tensor_id=800 + f)
        row["mult_then_trc_aby3_random_r"] = ctx.count_trunc_failures(64, f, pg, a0, a1)
        a0, a1 = ctx.trunc_aby3(64, f, p0, p1, tensor_id=800 + f, fixed_r=1 << f)
        row["mult_then_trc_aby3_fixed_r"] = ctx.count_trunc_failures(64, f, pg, a0, a1)
        s0, s1 = ctx.trunc_prob(64, f, p0, p1)
        row["mult_then_trc_secureml"] = ctx.count_trunc_failures(64, f, pg, s0, s1)
        t0, t1 = ctx.trunc_then_mul(64, f // 2, f - f // 2, x0, x1, y0, y1, tensor_id=900 + f)
        # trc-then-mult loses up to (|x| + |y|) / 2^(f/2) + 1 by design; count e1-scale misses
        rec = (t0.view(torch.int64) + t1.view(torch.int64)) - (pg >> f)
        row["trc_then_mult_e1_scale_errors"] = int((rec.abs() > (1 << 20)).sum().item())
        out[f"f={f}"] = row
    return out


def rss_bench(ctx, prm, buf, n):
    """Alg. drelu2 + the replicated ReLU product on 2-of-3 replicated shares
    of the same truncated product (components trc0, 0, trc1)."""
    import torch
    z = torch.zeros_like(buf["trc0"])
    ys = tuple(torch.empty_like(buf["trc0"]) for _ in range(3))
    for _ in range(3):
        ctx.rss_relu(prm, buf["trc0"], z, buf["trc1"], 4, out=ys)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        ctx.rss_relu(prm, buf["trc0"], z, buf["trc1"], 4, out=ys)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    return {"kernel_ms": ms, "elems_per_s": n / (ms / 1e3)}


def b1_pair(args, local, dev):
    """`--workload b1-pair`: one launch of each DReLU kernel on the same
    shares (magnitudes below 2^21, l = 64, lx = 24, c = 0), for profiling."""
    import torch
    from paper_2309_04909_gb300 import Context, Params, workloads as W
    ctx = Context(5, device=local)
    x = W.magnitude_bounded_ints(args.n, 21, seed=1)
    x0, x1 = ctx.share(64, torch.from_numpy(x).to(dev), 1)
    prm = Params(64, 24, 0)
    o = (torch.empty_like(x0), torch.empty_like(x1))
    ctx.drelu_b1(prm, x0, x1, 5, out=o)
    ctx.drelu(prm, x0, x1, 5, out=o)
    torch.cuda.synchronize()
    print(json.dumps({"workload": "b1-pair", "n": args.n}), flush=True)
    ctx.close()


def _parties3_worker(rank, port, out_dir, n, steps, warmup, transport="ipc"):
    """One party of `--workload parties3` (rank = party)."""
    import torch
    import torch.distributed as dist
    from paper_2309_04909_gb300 import Context, Params, workloads as W
    from paper_2309_04909_gb300.parties import (IpcTransport, PartyProcess, Transport,
                                                context_stages)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=3)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = Context(BASE_SEED)
    prm = Params(64, 24, 0)
    x = W.magnitude_bounded_ints(n, 21, seed=1)
    s0, s1 = ctx.share(64, torch.from_numpy(x).to(dev), 1)
    share = (s0, s1, None)[rank]

    def clock():
        torch.cuda.synchronize()
        return time.perf_counter()

    tr = IpcTransport(dev) if transport == "ipc" else Transport(dev, direct=False)
    pp = PartyProcess(rank, context_stages(ctx), tr, clock=clock)
    walls, out = [], None
    for i in range(warmup + steps):
        if i == warmup:
            pp.timing = {"compute": 0.0, "transport": 0.0}
            tr.sent = {}
        dist.barrier()
        t0 = time.perf_counter()
        out = pp.run(prm, True, share, n, 7)
        torch.cuda.synchronize()
        if i >= warmup:
            walls.append(time.perf_counter() - t0)
    wall = torch.tensor(walls, dtype=torch.float64)
    dist.all_reduce(wall, op=dist.ReduceOp.MAX)          # each step: its slowest party
    same = None
    if out is not None:
        f = ctx.relu(prm, s0, s1, tensor_id=7)
        same = bool(torch.equal(out, f[rank]))
    res = {"party": rank, "step_s": wall.tolist(), "compute_s": pp.timing["compute"] / steps,
           "transport_s": pp.timing["transport"] / steps,
           "sent_bytes_per_step": {f"{a}->{b}": v // steps for (a, b), v in tr.sent.items()},
           "identical_to_fused": same}
    with open(os.path.join(out_dir, f"p{rank}.json"), "w") as fh:
        json.dump(res, fh)
    del pp, tr
    torch.cuda.synchronize()
    dist.barrier()
    dist.destroy_process_group()
    ctx.close()


def parties3(args):
    """`--workload parties3`: the ReLU of --n elements (l = 64, lx = 24) with
    P0, P1 and P2 as three processes, each with its own context on GPU 0, every
    message moved into the receiver's memory: copied by the GPU into the
    receiver's device buffer (--party-transport ipc, CUDA IPC, with a token
    handshake over gloo) or through host memory by gloo.  One
    JSON line: elements/s over the slowest party's step time, each party's
    compute and transport time per step, the bytes each sent, and whether P0's
    and P1's outputs equal the fused kernel's."""
    import socket
    import torch.multiprocessing as mp
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_parties3_worker, nprocs=3, join=True, start_method="spawn",
                           args=(port, d, args.n, args.steps, args.warmup,
                                 args.party_transport))
        r = [json.load(open(os.path.join(d, f"p{k}.json"))) for k in range(3)]
    step_s = statistics.median(r[0]["step_s"])
    print(json.dumps({
        "metric": "relu elems/s, three party processes", "workload": "parties3",
        "value": args.n / step_s, "unit": "elems/s", "ms_per_step": step_s * 1e3,
        "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": f"ReLU, l=64 lx=24, n={args.n}, P0/P1/P2 as processes on one "
                               "GPU, " + ("messages copied by the GPU into the receiver's "
                                          "device memory (CUDA IPC), tokens over gloo"
                                          if args.party_transport == "ipc" else
                                          "gloo through host memory"),
                   "transport": args.party_transport},
        "parties": {f"P{x['party']}": {k: x[k] for k in ("compute_s", "transport_s",
                                                          "sent_bytes_per_step",
                                                          "identical_to_fused")} for x in r},
    }), flush=True)


def b1_bench(ctx, x0, x1, n, reps=20):
    """The Bicoptor 1.0-style protocol (SecureML truncations, recursive sums
    and masks in Z_{2^l}) against Bicoptor 2.0 on the same 2^22 shares at
    l = 64, at lx = 24 and at the paper's key bits lx = 7 (c = 24): kernel time
    and the bits each of P0 and P1 sends P2 per element."""
    import torch
    from paper_2309_04909_gb300 import Params
    out = {}
    o = (torch.empty_like(x0), torch.empty_like(x1))
    for lx, c in ((24, 0), (7, 24)):
        prm = Params(64, lx, c)
        row = {}
        for name, fn in (("b2_drelu", ctx.drelu), ("b2_relu", ctx.relu),
                         ("b1_drelu", ctx.drelu_b1), ("b1_relu", ctx.relu_b1)):
            for _ in range(3):
                fn(prm, x0, x1, 5, out=o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn(prm, x0, x1, 5, out=o)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[name] = {"kernel_ms": ms, "elems_per_s": n / (ms / 1e3)}
        row["bits_per_element_p0_to_p2"] = {"b2": (lx + 1) ** 2, "b1": (lx + 1) * 64}
        out[f"lx{lx}_c{c}"] = row
    return out


def parties_bench(ctx, prm, buf, n, fused_ms):
    """The same ReLU with each party's work in its own kernel and every
    message in a device buffer (bit-packed w at lx+1 bits per value): the
    communication path the fused kernel keeps in registers."""
    import torch
    msgs = ctx.party_buffers(prm, n)
    out = (torch.empty_like(buf["relu0"]), torch.empty_like(buf["relu1"]))
    for _ in range(3):
        ctx.relu_parties(prm, buf["trc0"], buf["trc1"], 4, out=out, msgs=msgs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        ctx.relu_parties(prm, buf["trc0"], buf["trc1"], 4, out=out, msgs=msgs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    same = bool(torch.equal(out[0], buf["relu0"]) and torch.equal(out[1], buf["relu1"]))
    msg_bytes = sum(t.numel() * t.element_size() for t in msgs.values())
    return {"kernel_ms": ms, "elems_per_s": n / (ms / 1e3), "vs_fused": fused_ms / ms,
            "message_bytes_per_element": msg_bytes / n,
            "protocol_bits_per_element_p0_to_p2": (prm.lx + 1) ** 2,
            "identical_to_fused": same, "launches": 3}


# The paper's measured throughput (ops/s) of its DReLU and ReLU at lx = 7 on
# three P100 servers, from its DReLU and ReLU tables (Sec. 7): context beside
# the projection below, another machine's numbers.
PAPER_OPS = {
    "drelu": {"LAN1": {"1e3": 1002646.99, "1e4": 7268181.36, "1e5": 17547892.59,
                       "1e6": 17062429.72},
              "LAN2": {"1e3": 713210.80, "1e4": 3898498.69, "1e5": 5863383.17,
                       "1e6": 4648006.47},
              "WAN": {"1e3": 23871.19, "1e4": 184700.86, "1e5": 430429.65, "1e6": 526221.62}},
    "relu": {"LAN1": {"1e3": 621596.76, "1e4": 4395585.07, "1e5": 10041441.03,
                      "1e6": 11088207.80},
             "LAN2": {"1e3": 426070.40, "1e4": 2174901.21, "1e5": 3197114.92,
                      "1e6": 2946653.78},
             "WAN": {"1e3": 12060.67, "1e4": 114435.72, "1e5": 192806.77, "1e6": 279506.84}},
}


def network_projection(sweep):
    """A model, not a measurement: the protocol at the paper's key width
    (lx = 7, l = 64) with each party on a GB300 and the messages on the
    paper's three networks.  gpu_ms is the measured time of the whole call
    with all three parties on one GPU (so an upper bound on any one party's
    work); net_ms is costmodel.network_seconds, the two rounds' latency and
    bits over the busiest link.  Projected ops/s = n / (gpu + net); the
    paper's measured figure on P100 servers is beside it."""
    from paper_2309_04909_gb300 import costmodel as C
    out = {}
    for op in ("drelu", "relu"):
        row = {}
        for net, (bw, rtt) in C.PAPER_NETWORKS.items():
            cells = {}
            for e in range(3, 7):
                key, n = f"1e{e}", 10 ** e
                gpu_s = sweep[f"{op}_lx7"][key]["ms"] / 1e3
                net_s = C.network_seconds(64, 7, n, op == "relu", bw, rtt)
                cells[key] = {"gpu_ms": gpu_s * 1e3, "net_ms": net_s * 1e3,
                              "projected_ops_per_s": n / (gpu_s + net_s),
                              "paper_ops_per_s": PAPER_OPS[op][net][key]}
            row[net] = cells
        out[op] = row
    out["model"] = ("one full-duplex link per server at the network's bandwidth each way; per "
                    "round half the round-trip time plus the busiest server's bits in or out; "
                    "w_j of (lx+1)^2 bits per element, openings, e, [c]_1 and the reply of l "
                    "bits; GPU time measured on one GB300 for all three parties")
    return out


def size_sweep(ctx, dev):
    """DReLU and ReLU against batch size on device-resident shares, l = 64:
    at the paper's key width lx = 7 (its unit-test setting) and at lx = 24.
    Ten calls are replayed from a CUDA graph, so the time is the GPU's (a
    launch of up to about 10^5 elements runs the four-lanes-per-element
    kernel); `eager_us_per_call` is the same call made from Python, whose
    host cost dominates at small batches."""
    import torch
    from paper_2309_04909_gb300 import Params
    from paper_2309_04909_gb300.batch import time_ms
    out = {}
    nmax = 10 ** 8
    g = torch.Generator(device=dev).manual_seed(5)
    s0 = torch.randint(-2**62, 2**62, (nmax,), device=dev, generator=g)
    s1 = torch.randint(-2**62, 2**62, (nmax,), device=dev, generator=g)
    o0, o1 = torch.empty_like(s0), torch.empty_like(s1)
    side = torch.cuda.Stream()
    for lx in (7, 24):
        prm = Params(64, lx, 0)
        for op in ("drelu", "relu"):
            fn = ctx.drelu if op == "drelu" else ctx.relu
            row = {}
            for e in range(3, 9):
                n = 10 ** e
                a, b, c, d = s0[:n], s1[:n], o0[:n], o1[:n]
                call = lambda: fn(prm, a, b, 5, out=(c, d))
                reps = 10 if e < 8 else 2
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):
                    call()
                torch.cuda.current_stream().wait_stream(side)
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    for _ in range(reps):
                        call()
                ms = time_ms(graph.replay, reps=3, warmup=1) / reps
                row[f"1e{e}"] = {"ms": ms, "elems_per_s": n / (ms / 1e3)}
                if e == 3:
                    row["eager_us_per_call"] = 1e3 * time_ms(call, reps=20, warmup=3)
            out[f"{op}_lx{lx}"] = row
    return out


def uniform_l32_drelu_check(ctx, dev):
    """DReLU of 65,536 uniform reals in [-1000, 1000] (f = 12) in
    Z_{2^32}, (lx, c) = (9, 14).  Checks every element against the oracle
    (bit-exact shares) and the reconstructed sign against the plaintext; every
    mismatch must lie in the predicted set |x| < 2^c or the band around
    xi* 2^c."""
    import torch
    import oracle as O
    from paper_2309_04909_gb300 import Params, workloads as W
    n, ring, lx, c = 65536, 32, 9, 14
    X = W.uniform_reals(n, -1000.0, 1000.0, seed=0)
    xi = np.rint(np.ldexp(X, 12)).astype(np.int64)
    s0, s1 = ctx.share(ring, torch.from_numpy(xi).to(dev), tensor_id=100)
    prm = Params(ring, lx, c)
    for _ in range(3):
        o0, o1 = ctx.drelu(prm, s0, s1, tensor_id=101)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(20):
        o0, o1 = ctx.drelu(prm, s0, s1, tensor_id=101, out=(o0, o1))
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / 20
    g0 = o0.cpu().numpy().view(np.uint32)
    g1 = o1.cpu().numpy().view(np.uint32)
    m = np.uint64(0xFFFFFFFF)
    e0, e1 = O.share(ring, xi.astype(np.uint64) & m, ctx.seed, 100)
    r0, r1 = O.drelu(O.params(ring, lx, c), e0, e1, ctx.seed, 101, threads=O.max_threads())
    parity_mismatch = int((g0 != r0).sum() + (g1 != r1).sum())
    drelu = (g0.astype(np.uint64) + g1.astype(np.uint64)) & m
    want = (xi >= 0).astype(np.uint64)
    bad = np.nonzero(drelu != want)[0]
    mags = np.abs(xi[bad])
    xi_star = [v for v in range(1, 1 << lx) if v + (v + 1) // 2 in ((1 << lx) - 1, 1 << lx)]
    predicted = (mags < (1 << c)) | np.any(
        [np.abs(mags - e * (1 << c)) < (1 << c) for e in xi_star], axis=0)
    return {"workload": "65,536 U[-1000,1000] reals, f=12, Z_2^32, (lx, c) = (9, 14), DReLU",
            "kernel_ms": ms, "elems_per_s": n / (ms / 1e3),
            "oracle_mismatches": parity_mismatch, "sign_mismatches": int(bad.size),
            "sign_mismatches_outside_predicted_set": int((~predicted).sum()) if bad.size else 0}


def serving_only(args):
    """The serving workload alone: Poisson 2,000 req/s for --serve-seconds,
    1-64 images per request, 50/50 LeNet / VGG-16 ReLU sets, l = 64, f = 16,
    40 GB admission budget, seed 4."""
    import torch
    from paper_2309_04909_gb300 import Context, Params, workloads as W
    from paper_2309_04909_gb300.serve import Engine, ServingSetup
    dev = torch.device("cuda", 0)
    ctx = Context(0xB1C0_5E12, device=0)
    budget = 40 << 30
    setup = ServingSetup(ctx, Params(64, 24, 0), budget, seed=4, pool_images=64)
    trace = W.serving_trace(2000.0, args.serve_seconds, seed=4)
    reqs = setup.requests_from_trace(trace)
    st = Engine(setup.executor(schedule=1), budget, max_iter_elems=1 << 24).run(reqs)
    s = st.summary()
    s.update({"metric": METRIC, "workload": f"serving: Poisson 2000 req/s x {args.serve_seconds} s, "
                                            "1-64 images, LeNet/VGG-16 50/50, l=64 f=16",
              "offered_elems_per_s": sum(r.elements for r in reqs) / args.serve_seconds})
    print(json.dumps(s), flush=True)
    ctx.close()


def serving_bench(ctx, dev, capacity, seconds, load_seconds, bvp, budget=40 << 30):
    """Continuous-batching serving: Poisson arrivals of 1-64-image LeNet /
    VGG-16 ReLU requests (50/50), l = 64, under a 40 GB admission budget.
    Runs the offered 2,000 req/s and 50 % / 90 % of the measured batched
    capacity, each for `seconds` of arrivals; reports p50/p99 latency."""
    from paper_2309_04909_gb300 import Params, workloads as W
    from paper_2309_04909_gb300.serve import Engine, ServingSetup, ideal_latencies
    prm = Params(64, 24, 0)
    setup = ServingSetup(ctx, prm, budget, seed=4, pool_images=64)
    mean_elems = 0.5 * 32.5 * (setup.per_image["vgg16"] + setup.per_image["lenet"])
    sched = 1 if bvp.get("schedule") == "grid" else 0
    out = {"budget_bytes": budget, "mean_elems_per_request": mean_elems,
           "capacity_elems_per_s": capacity}
    for label, rate in (("offered_2000_rps", 2000.0),
                        ("load_90pct", 0.9 * capacity / mean_elems),
                        ("load_50pct", 0.5 * capacity / mean_elems)):
        window = seconds if label.startswith("offered") else load_seconds
        trace = W.serving_trace(rate, window, seed=4)
        reqs = setup.requests_from_trace(trace)
        st = Engine(setup.executor(schedule=sched), budget, max_iter_elems=1 << 24).run(reqs)
        s = st.summary()
        # the yardstick: the same arrivals on an ideal first-come server of the
        # measured capacity (no iteration quantum, no launch cost)
        ideal = sorted(ideal_latencies([r.arrival_s for r in trace],
                                       [r.images * setup.per_image[r.net] / capacity
                                        for r in trace], "fcfs"))
        s["ideal_fcfs_ms"] = {"p50": 1e3 * ideal[len(ideal) // 2],
                              "p99": 1e3 * ideal[min(len(ideal) - 1, int(0.99 * len(ideal)))]}
        s["arrival_window_s"] = window
        s["rate_rps"] = rate
        s["offered_elems_per_s"] = rate * mean_elems
        out[label] = s
    return out


if __name__ == "__main__":
    main()
