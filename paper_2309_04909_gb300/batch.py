"""Batched ReLU over many tensors: one persistent launch over a tile queue.

A network's ReLU layers (and many inferences of uneven size) are planned once
into a tile table (bc_relu_batch_plan) and run as a single persistent kernel
(bc_relu_batch_run) whose CTAs pull tiles from an atomic counter.  The run is
stream-capturable, so a ReluBatch can be replayed through a CUDA graph.
The autotuner picks the schedule, the elements per thread (grid schedule), the
tile size and CTAs per SM (persistent schedule) and the unroll of the key-bit
loop by timing the candidates on the actual tensors; its choice is cached per
(tensor mix, GPU).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence, Tuple

import torch

from . import Context, Params

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

TILE_CANDIDATES = (128, 256, 512, 1024, 2048)
EPT_CANDIDATES = (1, 2, 4)
UNROLL_CANDIDATES = (0, 2, 3)   # 0: the whole key-bit loop
# The launch shape the kernels are tuned and profiled for: grid schedule,
# 256-element tiles, one element per thread, the key-bit loop unrolled whole.
DEFAULT_LAUNCH = {"schedule": 1, "tile_elems": 256, "ctas_per_sm": 0, "elems_per_thread": 1,
                  "slot_unroll": 0}
# Another candidate replaces the default only when it is faster by more than
# this fraction, so that timing noise between near-equal shapes does not flip
# the choice from run to run.
PREFER_DEFAULT_WITHIN = 0.01


class ReluBatch:
    """items: (Params, s0, s1, o0, o1, tensor_id[, op]) per tensor."""

    def __init__(self, ctx: Context, items: Sequence[Tuple], tile_elems: int = 0,
                 ctas_per_sm: int = 0, schedule: int = 0, elems_per_thread: int = 0,
                 slot_unroll: int = 0):
        self.ctx = ctx
        self.items = list(items)
        self.tile_elems = tile_elems
        self.ctas_per_sm = ctas_per_sm
        self.schedule = schedule
        self.elems_per_thread = elems_per_thread
        self.slot_unroll = slot_unroll
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.plan()

    @property
    def elements(self) -> int:
        return int(sum(it[1].numel() for it in self.items))

    def plan(self):
        self.ctx.relu_batch_plan(self.items, self.tile_elems, self.ctas_per_sm, self.schedule,
                                 self.elems_per_thread, self.slot_unroll)
        self.graph = None

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.ctx.relu_batch_run()

    def capture(self):
        """Capture one run in a CUDA graph; later run() calls replay it."""
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):          # warm the stream before capture
            self.ctx.relu_batch_run()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.ctx.relu_batch_run()
        torch.cuda.synchronize()
        self.graph = g

    def status(self) -> int:
        return self.ctx.batch_status()


def time_ms(fn, reps: int = 5, warmup: int = 2) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def _mix_key(items) -> str:
    rings = sorted({(it[0].ring_bits, it[0].lx) for it in items})
    total = sum(it[1].numel() for it in items)
    return (f"v4|{torch.cuda.get_device_name()}|{rings}|n~2^{max(total, 1).bit_length()}"
            f"|t{len(items)}")


def autotune(ctx: Context, items: Sequence[Tuple], reps: int = 3,
             use_cache: bool = True) -> Dict[str, float]:
    """Time the candidates on `items` and return the best {"schedule",
    "tile_elems", "ctas_per_sm", "elems_per_thread", "slot_unroll", "ms"}:
    the grid schedule at every (elements per thread, key-bit unroll), then
    the persistent schedule at every (tile, CTAs per SM) with the best
    unroll.  DEFAULT_LAUNCH is kept unless the best candidate beats it by more
    than PREFER_DEFAULT_WITHIN.  Outputs of the tensors are written (the
    protocol is deterministic, so reruns give identical results)."""
    key = _mix_key(items)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    best = None
    timed = {}

    def consider(cfg):
        nonlocal best
        b = ReluBatch(ctx, items, cfg["tile_elems"], cfg["ctas_per_sm"], cfg["schedule"],
                      cfg["elems_per_thread"], cfg["slot_unroll"])
        ms = time_ms(b.run, reps=reps, warmup=1)
        timed[tuple(sorted(cfg.items()))] = ms
        if best is None or ms < best["ms"]:
            best = dict(cfg, ms=ms)

    for ept in EPT_CANDIDATES:
        for u in UNROLL_CANDIDATES:
            consider({"schedule": 1, "tile_elems": 256 * ept, "ctas_per_sm": 0,
                      "elems_per_thread": ept, "slot_unroll": u})
    u = best["slot_unroll"]
    for tile in TILE_CANDIDATES:
        for cps in (0, 1, 2, 3):
            consider({"schedule": 0, "tile_elems": tile, "ctas_per_sm": cps,
                      "elems_per_thread": 1, "slot_unroll": u})
    d_ms = timed.get(tuple(sorted(DEFAULT_LAUNCH.items())))
    if d_ms is not None and d_ms <= best["ms"] * (1.0 + PREFER_DEFAULT_WITHIN):
        best = dict(DEFAULT_LAUNCH, ms=d_ms)
    cache[key] = best
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        json.dump(cache, open(_CACHE, "w"), indent=1)
    except OSError:
        pass
    return best
