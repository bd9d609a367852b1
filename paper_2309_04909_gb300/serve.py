"""Serving loop: continuous batching of private-inference ReLU requests.

Requests (a private-inference activation batch: the ReLU tensors of 1..64
images of a LeNet- or VGG-16-shaped network, secret-shared in Z_{2^64}) arrive
over time.  The loop admits a request as soon as it has arrived and its
output shares fit in the device-memory budget, and every scheduler iteration
launches ONE batched DReLU/ReLU call (the persistent/grid batch kernel of the
library) over the next chunks of all admitted requests.  Requests that arrive
while others are on the GPU join the next iteration, so their work overlaps on
the device; a finished request frees its memory at once.  Up to `max_inflight`
iterations are queued on the stream while the host plans the next one.

A request is one flattened tensor keyed by its own tensor id; a chunk carries
its element offset, so every element gets the randomness it would get alone:
a request's result is bit-identical alone and in the mix.

Randomness (masks, shuffles, Beaver triples) is derived from the pre-shared
seeds inside the kernel, so the device-memory budget covers the input and
output shares only: 32 bytes per element at l = 64.  A request larger than
the whole budget is rejected.
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import time
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple


# ---------------------------------------------------------------------------
# Device arena: first-fit allocation with coalescing, in bytes (host logic).
# ---------------------------------------------------------------------------

class Arena:
    """First-fit allocator over [0, capacity) with 256-byte alignment."""

    ALIGN = 256

    def __init__(self, capacity: int):
        self.capacity = capacity
        self._free: List[Tuple[int, int]] = [(0, capacity)]   # sorted (offset, size)
        self.used = 0
        self.peak = 0

    def alloc(self, size: int) -> Optional[int]:
        size = (size + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (off, sz) in enumerate(self._free):
            if sz >= size:
                if sz == size:
                    self._free.pop(i)
                else:
                    self._free[i] = (off + size, sz - size)
                self.used += size
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off: int, size: int) -> None:
        size = (size + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        i = bisect.bisect_left(self._free, (off, 0))
        self._free.insert(i, (off, size))
        self.used -= size
        # coalesce with neighbours
        if i + 1 < len(self._free) and self._free[i][0] + self._free[i][1] == self._free[i + 1][0]:
            self._free[i] = (self._free[i][0], self._free[i][1] + self._free[i + 1][1])
            self._free.pop(i + 1)
        if i > 0 and self._free[i - 1][0] + self._free[i - 1][1] == self._free[i][0]:
            self._free[i - 1] = (self._free[i - 1][0], self._free[i - 1][1] + self._free[i][1])
            self._free.pop(i)

    @property
    def free_blocks(self) -> int:
        return len(self._free)


# ---------------------------------------------------------------------------
# Requests and the scheduler
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    elements: int
    net: str = ""
    images: int = 0
    # filled by the engine
    offset: Optional[int] = None        # arena offset (bytes) of the request's shares
    rejected: bool = False
    done: int = 0                       # elements launched so far
    retired: int = 0                    # elements whose iteration finished
    admitted_s: Optional[float] = None
    finished_s: Optional[float] = None
    # optional client limits on the engine clock (seconds): a request not
    # finished by its deadline expires, one past cancel_at_s is cancelled
    deadline_s: Optional[float] = None
    cancel_at_s: Optional[float] = None
    dropped: Optional[str] = None       # "expired" or "cancelled"

    @property
    def latency_s(self) -> Optional[float]:
        if self.finished_s is None:
            return None
        return self.finished_s - self.arrival_s


@dataclasses.dataclass
class Chunk:
    req: ServeRequest
    start: int          # first element of the chunk within the request
    count: int


class Executor:
    """What the engine needs from the device: bytes per element of output,
    launching one iteration, and polling it.  `launch` returns a handle whose
    `done()` says whether the iteration finished and whose `finish_s()` gives
    its completion time on the engine clock."""

    bytes_per_element: int = 32      # input + output shares, both parties, l = 64

    def launch(self, chunks: Sequence[Chunk]):
        raise NotImplementedError

    def now(self) -> float:
        raise NotImplementedError

    def wait(self, handle) -> None:
        raise NotImplementedError

    def sleep_until(self, t: float) -> None:
        raise NotImplementedError


@dataclasses.dataclass
class ServeStats:
    requests: int
    completed: int
    elements: int
    wall_s: float
    latencies_s: List[float]
    iterations: int
    peak_bytes: int
    max_waiting: int
    rejected: int = 0
    expired: int = 0
    cancelled: int = 0
    # the queue when the last request arrives: requests waiting for admission
    # or admitted and unfinished, and the elements finished by then
    arrival_end_s: float = 0.0
    backlog_at_arrival_end: int = 0
    elements_by_arrival_end: int = 0

    def summary(self) -> Dict[str, float]:
        lat = sorted(self.latencies_s)

        def pct(q):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]

        # latency histogram: counts per power-of-two bucket of milliseconds,
        # keyed by the bucket's upper edge ("<=1", "<=2", ..., ">1024")
        hist: Dict[str, int] = {}
        for v in lat:
            ms, edge = 1e3 * v, 1.0
            while ms > edge and edge <= 1024.0:
                edge *= 2.0
            key = f"<={edge:g}" if edge <= 1024.0 else ">1024"
            hist[key] = hist.get(key, 0) + 1
        return {"requests": self.requests, "completed": self.completed,
                "elements": self.elements, "wall_s": self.wall_s,
                "elems_per_s": self.elements / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": None if not lat else 1e3 * pct(0.50),
                "p99_ms": None if not lat else 1e3 * pct(0.99),
                "max_ms": None if not lat else 1e3 * lat[-1],
                "latency_histogram_ms": hist,
                "iterations": self.iterations, "peak_bytes": self.peak_bytes,
                "max_waiting": self.max_waiting, "rejected": self.rejected,
                "expired": self.expired, "cancelled": self.cancelled,
                "arrival_end_s": self.arrival_end_s,
                "backlog_at_arrival_end": self.backlog_at_arrival_end,
                "queue_growth_per_s": (self.backlog_at_arrival_end / self.arrival_end_s
                                       if self.arrival_end_s > 0 else 0.0),
                "elems_per_s_during_arrivals": (self.elements_by_arrival_end
                                                / self.arrival_end_s
                                                if self.arrival_end_s > 0 else 0.0),
                "drain_s": self.wall_s - self.arrival_end_s}


class Engine:
    """Continuous-batching scheduler (host side; the executor runs the GPU)."""

    def __init__(self, executor: Executor, budget_bytes: int, max_iter_elems: int = 1 << 24,
                 max_inflight: int = 2, min_chunk: int = 1 << 16, max_share: int = 8):
        self.ex = executor
        self.arena = Arena(budget_bytes)
        self.max_iter_elems = max_iter_elems
        self.max_inflight = max_inflight
        self.min_chunk = min_chunk
        self.max_share = max_share

    def _plan_iteration(self, active: List[ServeRequest]) -> List[Chunk]:
        """Fair share among the `max_share` oldest admitted requests with work
        left: each gets an equal quantum of the iteration (small requests
        finish in their first iteration); what the quanta leave unused goes
        to the oldest requests first."""
        live = [r for r in active if r.elements > r.done and r.dropped is None][:self.max_share]
        if not live:
            return []
        budget = self.max_iter_elems
        quantum = max(budget // len(live), self.min_chunk)
        take: Dict[int, int] = {}
        for r in live:
            if budget == 0:
                break
            t = min(r.elements - r.done, quantum, budget)
            take[r.rid] = t
            budget -= t
        for r in live:
            if budget == 0:
                break
            extra = min(r.elements - r.done - take.get(r.rid, 0), budget)
            if extra > 0:
                take[r.rid] = take.get(r.rid, 0) + extra
                budget -= extra
        chunks = []
        for r in live:
            t = take.get(r.rid, 0)
            if t:
                chunks.append(Chunk(r, r.done, t))
                r.done += t
        return chunks

    def run(self, requests: Sequence[ServeRequest],
            on_complete: Optional[Callable[[ServeRequest], None]] = None) -> ServeStats:
        """Serve `requests` to completion.  `on_complete(req)` runs when a
        request's last iteration has finished, before its memory is freed
        (work it queues on the stream is ordered before any reuse)."""
        pending: Deque[ServeRequest] = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: Deque[ServeRequest] = collections.deque()
        active: List[ServeRequest] = []
        inflight: Deque[Tuple[object, List[Chunk]]] = collections.deque()
        out_b = self.ex.bytes_per_element
        iterations, max_waiting, done_elems, rejected = 0, 0, 0, 0
        arrival_end, backlog_end, elems_end = 0.0, 0, 0
        t0 = self.ex.now()
        while pending or waiting or active or inflight:
            now = self.ex.now() - t0
            while pending and pending[0].arrival_s <= now:
                r = pending.popleft()
                if r.elements * out_b > self.arena.capacity:
                    r.rejected = True
                    rejected += 1
                else:
                    waiting.append(r)
                if not pending:          # the last arrival: note the queue
                    arrival_end = r.arrival_s
                    backlog_end = len(waiting) + sum(1 for a in active
                                                     if a.finished_s is None)
                    elems_end = done_elems
            max_waiting = max(max_waiting, len(waiting))
            # client limits: drop queued requests at once; an admitted one
            # stops getting chunks and is freed when its chunks in flight retire
            for r in list(waiting) + active:
                if r.dropped is None:
                    if r.cancel_at_s is not None and now >= r.cancel_at_s:
                        r.dropped = "cancelled"
                    elif r.deadline_s is not None and now >= r.deadline_s:
                        r.dropped = "expired"
            if any(r.dropped for r in waiting):
                waiting = collections.deque(r for r in waiting if r.dropped is None)
            # admission: FIFO while the output shares fit in the budget
            while waiting:
                r = waiting[0]
                off = self.arena.alloc(r.elements * out_b)
                if off is None:
                    break
                r.offset, r.admitted_s = off, now
                active.append(waiting.popleft())
            # retire finished iterations in order
            progressed = False
            while inflight and inflight[0][0].done():
                handle, chunks = inflight.popleft()
                fin = handle.finish_s() - t0
                for c in chunks:
                    c.req.retired += c.count
                    done_elems += c.count
                    if c.req.retired == c.req.elements:
                        c.req.finished_s = fin
                        if on_complete is not None:
                            on_complete(c.req)
                        self.arena.free(c.req.offset, c.req.elements * out_b)
                progressed = True
            # a dropped request leaves once nothing of it is in flight
            keep = []
            for r in active:
                if r.dropped is not None and r.retired == r.done and r.finished_s is None:
                    self.arena.free(r.offset, r.elements * out_b)
                    r.offset = None
                    progressed = True
                elif r.retired < r.elements and not (r.dropped is not None and r.offset is None):
                    keep.append(r)
            active = keep
            # launch the next iteration over the admitted requests' next chunks
            if len(inflight) < self.max_inflight:
                chunks = self._plan_iteration(active)
                if chunks:
                    inflight.append((self.ex.launch(chunks), chunks))
                    iterations += 1
                    continue
            if not progressed:
                if inflight:
                    self.ex.wait(inflight[0][0])
                elif pending and not waiting:
                    self.ex.sleep_until(t0 + pending[0].arrival_s)
        wall = self.ex.now() - t0
        lat = [r.latency_s for r in requests if r.latency_s is not None]
        expired = sum(1 for r in requests if r.dropped == "expired" and r.finished_s is None)
        cancelled = sum(1 for r in requests if r.dropped == "cancelled" and r.finished_s is None)
        return ServeStats(len(requests), len(lat), done_elems, wall, lat, iterations,
                          self.arena.peak, max_waiting, rejected, expired, cancelled,
                          arrival_end, backlog_end, elems_end)


# ---------------------------------------------------------------------------
# Executors
# ---------------------------------------------------------------------------

def ideal_latencies(arrivals_s: Sequence[float], service_s: Sequence[float],
                    policy: str = "fcfs") -> List[float]:
    """Latencies (completion - arrival) of the requests on an ideal single
    server: no launch cost, instant preemption, work `service_s` seconds each.
    policy: "fcfs" (first come, first served), "ps" (processor sharing: every
    unfinished request served at an equal share) or "srpt" (shortest
    remaining work first).  The yardstick for the engine's tail: the same
    arrivals and sizes, with none of its iteration quantum or launch costs."""
    n = len(arrivals_s)
    order = sorted(range(n), key=lambda i: arrivals_s[i])
    arr = [float(arrivals_s[i]) for i in order]
    size = [float(service_s[i]) for i in order]
    done = [0.0] * n
    if policy == "fcfs":
        t = 0.0
        for i in range(n):
            t = max(t, arr[i]) + size[i]
            done[i] = t
    elif policy in ("ps", "srpt"):
        t, i, active = 0.0, 0, {}
        while i < n or active:
            if not active:
                t = max(t, arr[i])
                active[i] = size[i]
                i += 1
                continue
            k = len(active)
            if policy == "ps":
                dt_finish = min(active.values()) * k
            else:
                j = min(active, key=active.get)
                dt_finish = active[j]
            dt_arr = arr[i] - t if i < n else float("inf")
            dt = min(dt_finish, dt_arr)
            if policy == "ps":
                for j in active:
                    active[j] -= dt / k
            else:
                active[j] -= dt
            t += dt
            for j in [j for j, v in active.items() if v <= 1e-15]:
                done[j] = t
                del active[j]
            if dt_arr <= dt_finish and i < n:
                active[i] = size[i]
                i += 1
    else:
        raise ValueError(f"unknown policy {policy!r}")
    out = [0.0] * n
    for pos, i in enumerate(order):
        out[i] = done[pos] - arr[pos]
    return out


class FakeExecutor(Executor):
    """A simulated device for host-logic tests: an iteration of n elements
    takes n / rate seconds of simulated time, iterations run back to back."""

    def __init__(self, rate_elems_per_s: float, bytes_per_element: int = 32):
        self.rate = rate_elems_per_s
        self.bytes_per_element = bytes_per_element
        self.t = 0.0
        self.device_free_at = 0.0
        self.launched: List[List[Tuple[int, int, int]]] = []

    class _H:
        def __init__(self, ex, end):
            self.ex, self.end = ex, end

        def done(self):
            return self.ex.t >= self.end

        def finish_s(self):
            return self.end

    def now(self):
        return self.t

    def launch(self, chunks):
        n = sum(c.count for c in chunks)
        start = max(self.t, self.device_free_at)
        self.device_free_at = start + n / self.rate
        self.launched.append([(c.req.rid, c.start, c.count) for c in chunks])
        return FakeExecutor._H(self, self.device_free_at)

    def wait(self, handle):
        self.t = max(self.t, handle.end)

    def sleep_until(self, t):
        self.t = max(self.t, t)


class GpuExecutor(Executor):
    """Runs each iteration as one batched ReLU launch through the C-ABI.

    Inputs come from a device-resident pool of input shares; request r's
    element j reads pool element (pool_base(r) + j).  Its output shares go to
    out0/out1 at element slot offset // 32 + j: the arena accounts 32 bytes
    per element (the request's input and output shares), and out0/out1 hold
    budget / 32 slots each.  Completion times come from CUDA events on the
    launching stream, measured against an event recorded at construction."""

    def __init__(self, ctx, params, pool0, pool1, arena_tensor0, arena_tensor1,
                 pool_base: Callable[[ServeRequest], int], tensor_id: Callable[[ServeRequest], int],
                 schedule: int = 1, tile_elems: int = 0):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.prm = params
        self.pool0, self.pool1 = pool0, pool1
        self.out0, self.out1 = arena_tensor0, arena_tensor1   # int64 lanes, one per element slot
        self.pool_base = pool_base
        self.tensor_id = tensor_id
        self.schedule = schedule
        self.tile_elems = tile_elems
        self.prm_c = params.c_struct()
        self.bytes_per_element = 32
        if params.ring_bits <= 32:
            raise ValueError("the serving pool holds 64-bit lanes (l > 32)")
        self.t_host0 = time.perf_counter()
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev0.record()

    class _H:
        def __init__(self, ex, ev):
            self.ex, self.ev = ex, ev

        def done(self):
            return self.ev.query()

        def finish_s(self):
            return self.ex.ev0.elapsed_time(self.ev) / 1e3

    def now(self):
        return time.perf_counter() - self.t_host0

    def launch(self, chunks):
        from ._native import TensorDesc
        n = len(chunks)
        arr = (TensorDesc * n)()
        p0, p1 = self.pool0.data_ptr(), self.pool1.data_ptr()
        q0, q1 = self.out0.data_ptr(), self.out1.data_ptr()
        prm = self.prm_c
        for j, c in enumerate(chunks):
            ib = 8 * (self.pool_base(c.req) + c.start)
            ob = 8 * (c.req.offset // 32 + c.start)
            arr[j] = TensorDesc(p0 + ib, p1 + ib, q0 + ob, q1 + ob, c.count,
                                self.tensor_id(c.req), 0, prm, c.start)
        self.ctx.relu_batch_plan_descs(arr, n, tile_elems=self.tile_elems,
                                       schedule=self.schedule)
        self.ctx.relu_batch_run()
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record()
        return GpuExecutor._H(self, ev)

    def wait(self, handle):
        handle.ev.synchronize()

    def sleep_until(self, t):
        d = t - self.now()
        if d > 0:
            time.sleep(min(d, 0.01))


# ---------------------------------------------------------------------------
# GPU set-up for the LeNet / VGG-16 serving workload
# ---------------------------------------------------------------------------

class ServingSetup:
    """Device-resident input pool and output arena for serving runs.

    The pool holds the secret-shared activations of `pool_images` seeded
    images of each network (VGG-16 32x32 and LeNet 28x28 ReLU sets), laid out
    image-major, so a request of k images reads the pool prefix of k images
    of its network.  The arena holds budget / 32 element slots per output
    share array."""

    def __init__(self, ctx, params, budget_bytes: int, seed: int, pool_images: int = 64,
                 frac_bits: int = 16, tensor_id_base: int = 0x40000000):
        import numpy as np
        import torch

        from . import workloads as W
        self.ctx = ctx
        self.prm = params
        self.budget = budget_bytes
        self.per_image = {"vgg16": sum(W.VGG16_32_LAYERS), "lenet": sum(W.LENET_28_LAYERS)}
        parts, self.base = [], {}
        off = 0
        for net, layers in (("vgg16", W.VGG16_32_LAYERS), ("lenet", W.LENET_28_LAYERS)):
            self.base[net] = off
            g = np.random.Generator(np.random.PCG64([seed, 11, len(parts)]))
            sig = g.uniform(0.5, 8.0, size=len(layers))
            for _ in range(pool_images):
                for li, sz in enumerate(layers):
                    parts.append(np.rint(np.ldexp(g.normal(0.0, sig[li], size=sz), frac_bits))
                                 .astype(np.int64))
            off += pool_images * self.per_image[net]
        allx = torch.from_numpy(np.concatenate(parts)).to(ctx.device)
        self.pool0, self.pool1 = ctx.share(params.ring_bits, allx, tensor_id=0x3FFFFFFF)
        slots = budget_bytes // 32
        self.out0 = torch.empty(slots, dtype=torch.int64, device=ctx.device)
        self.out1 = torch.empty(slots, dtype=torch.int64, device=ctx.device)
        self.tid_base = tensor_id_base
        torch.cuda.synchronize()

    def requests_from_trace(self, trace) -> List[ServeRequest]:
        return [ServeRequest(r.rid, r.arrival_s, r.images * self.per_image[r.net], r.net, r.images)
                for r in trace]

    def tensor_id(self, r: ServeRequest) -> int:
        return self.tid_base + r.rid

    def executor(self, schedule: int = 1, tile_elems: int = 0) -> GpuExecutor:
        return GpuExecutor(self.ctx, self.prm, self.pool0, self.pool1, self.out0, self.out1,
                           pool_base=lambda r: self.base[r.net], tensor_id=self.tensor_id,
                           schedule=schedule, tile_elems=tile_elems)

    def outputs(self, r: ServeRequest):
        o = r.offset // 32
        return self.out0[o:o + r.elements], self.out1[o:o + r.elements]

    def inputs(self, r: ServeRequest):
        b = self.base[r.net]
        return self.pool0[b:b + r.elements], self.pool1[b:b + r.elements]
