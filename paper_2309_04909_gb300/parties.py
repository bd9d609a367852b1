"""P0, P1 and P2 as separate processes (Alg. drelu, Alg. relu of the UBL
protocol, each party on its own context and, with NCCL, its own GPU).

Every party runs only its own stages of the party-separated protocol
(bc_party_local / bc_party_helper / bc_party_finish) and every message is
moved into the receiver's own memory before the receiver's stage reads it:

  round 1   P0 -> P2  w0 (packed, (lx+1)^2 bits per element)
            P1 -> P2  w1
            P0 <-> P1 the openings [x]_j - [a]_j                     (ReLU)
  round 2   P2 -> P1  reply: [DReLU']_1 (DReLU) / e = DReLU' - b (ReLU)
            P2 -> P0  e                                              (ReLU)
            P2 -> P1  [c]_1, the preprocessing of the triple         (ReLU)

The transport is torch.distributed point-to-point: with NCCL (one process per
GPU) device tensors go straight into the receiver's device memory; with gloo
they travel through host memory (sender copies to the host, receiver copies
its received host buffer to its device).  No kernel of one party waits on
another party: each stage is launched only once its inputs have arrived.
The pre-shared seeds of Sec. 2.1 are the contexts' common 64-bit seed.
"""
from __future__ import annotations

import collections
import dataclasses
from typing import Dict, Optional, Tuple

import torch
import torch.distributed as dist

P0, P1, P2 = 0, 1, 2
# message tags (one per message kind, so that the order of different kinds
# between the same two parties never matters)
TAG_W, TAG_OPEN, TAG_REPLY, TAG_PRE = 11, 12, 13, 14


class Transport:
    """Point-to-point messages between the parties' ranks.  `direct`: the
    backend carries device tensors (NCCL); otherwise (gloo) messages are
    staged through host memory.  Bytes are counted per (sender, receiver)."""

    def __init__(self, device: torch.device, direct: bool, ranks=(0, 1, 2)):
        self.device = device
        self.direct = direct
        self.ranks = ranks
        self.sent: Dict[Tuple[int, int], int] = {}

    def _rank(self, party: int) -> int:
        return self.ranks[party]

    def isend(self, t: torch.Tensor, src: int, dst: int, tag: int):
        self.sent[(src, dst)] = self.sent.get((src, dst), 0) + t.numel() * t.element_size()
        payload = t if self.direct else t.cpu()
        return dist.isend(payload.contiguous(), self._rank(dst), tag=tag), payload

    def irecv(self, like: torch.Tensor, src: int, tag: int):
        buf = torch.empty_like(like) if self.direct else torch.empty(like.shape, dtype=like.dtype)
        return dist.irecv(buf, self._rank(src), tag=tag), buf

    def to_device(self, buf: torch.Tensor) -> torch.Tensor:
        return buf if self.direct else buf.to(self.device, non_blocking=False)

    def prepare(self, me: int, nbytes: Dict[int, int]) -> None:
        """Called by every party before a call's messages, with the same
        sizes (bytes per message kind); nothing to do for this transport."""


class _Deferred:
    """A request whose work runs when it is waited for."""

    def __init__(self, fn):
        self.fn = fn
        self.done = False

    def wait(self):
        if not self.done:
            self.fn()
            self.done = True
        return True


class IpcTransport(Transport):
    """Messages copied by the GPU straight into the receiver's own device
    memory (CUDA IPC between the parties' processes on one GPU).

    prepare() allocates this party's receive buffer per (sender, message
    kind) and maps every other party's through their IPC handles, exchanged
    once over the process group.  A message then takes a handshake of two
    one-word tokens through the process group:
      receiver  irecv(): waits for its own stream (its earlier stages are done
                with the buffer), tells the sender READY, and later waits for
                DATA before its stage reads the buffer;
      sender    isend(), when waited for: waits for READY, copies the message
                into the receiver's buffer on its stream, waits for the copy,
                then sends DATA.
    So no kernel of one party waits on another (each stage launches after its
    inputs have landed), and a buffer is never overwritten while it is read."""

    def __init__(self, device: torch.device, ranks=(0, 1, 2), group=None):
        super().__init__(device, direct=True, ranks=ranks)
        self.group = group
        self.own: Dict[Tuple[int, int], torch.Tensor] = {}      # (src, tag) -> my buffer
        self.remote: Dict[Tuple[int, int], torch.Tensor] = {}   # (dst, tag) -> its buffer
        self.sizes: Dict[int, int] = {}
        self._keep = collections.deque(maxlen=64)   # tokens of the requests in flight

    def prepare(self, me: int, nbytes: Dict[int, int]) -> None:
        from torch.multiprocessing.reductions import rebuild_cuda_tensor, reduce_tensor
        if all(self.sizes.get(t, -1) >= b for t, b in nbytes.items()):
            return
        self.own.clear()
        self.remote.clear()
        self.sizes = dict(nbytes)
        mine = {}
        for src in (P0, P1, P2):
            if src == me:
                continue
            for tag, nb in nbytes.items():
                buf = torch.empty(max(nb, 16), dtype=torch.uint8, device=self.device)
                self.own[(src, tag)] = buf
                mine[(src, me, tag)] = reduce_tensor(buf)[1]
        torch.cuda.synchronize(self.device)
        parts = [None, None, None]
        dist.all_gather_object(parts, mine, group=self.group)
        for part in parts:
            for (src, dst, tag), args in part.items():
                if src == me:
                    self.remote[(dst, tag)] = rebuild_cuda_tensor(*args)

    def _token(self):
        t = torch.ones(1, dtype=torch.int32)
        self._keep.append(t)
        return t

    def isend(self, t: torch.Tensor, src: int, dst: int, tag: int):
        nb = t.numel() * t.element_size()
        self.sent[(src, dst)] = self.sent.get((src, dst), 0) + nb
        target = self.remote[(dst, tag)]
        if nb > target.numel():
            raise ValueError("message larger than the receiver's prepared buffer")
        flat = t.contiguous().view(-1).view(torch.uint8)
        ready = self._token()
        r_ready = dist.irecv(ready, self._rank(dst), tag=2 * tag, group=self.group)

        def go():
            r_ready.wait()
            target[:nb].copy_(flat)
            torch.cuda.current_stream(self.device).synchronize()
            dist.isend(self._token(), self._rank(dst), tag=2 * tag + 1, group=self.group).wait()

        return _Deferred(go), t

    def irecv(self, like: torch.Tensor, src: int, tag: int):
        nb = like.numel() * like.element_size()
        own = self.own[(src, tag)]
        if nb > own.numel():
            raise ValueError("message larger than the prepared buffer")
        buf = own[:nb].view(like.dtype).view(like.shape)
        torch.cuda.current_stream(self.device).synchronize()
        r_data = dist.irecv(self._token(), self._rank(src), tag=2 * tag + 1, group=self.group)
        w_ready = dist.isend(self._token(), self._rank(src), tag=2 * tag, group=self.group)

        def done():
            w_ready.wait()
            r_data.wait()

        return _Deferred(done), buf

    def to_device(self, buf: torch.Tensor) -> torch.Tensor:
        return buf


def wait_all(reqs):
    for r in reqs:
        r.wait()


@dataclasses.dataclass
class Stages:
    """The three stage calls of one party (a Context's bc_party_* entry
    points); tests may substitute their own."""
    local: object
    helper: object
    finish: object
    buffers: object


def context_stages(ctx) -> Stages:
    return Stages(ctx.party_local, ctx.party_helper, ctx.party_finish, ctx.party_stage_buffers)


def message_sizes(buf: Dict[str, torch.Tensor]) -> Dict[int, int]:
    """Bytes of each message kind of one call, from a party's stage buffers."""
    nb = lambda k: buf[k].numel() * buf[k].element_size()
    return {TAG_W: nb("w"), TAG_OPEN: nb("open"), TAG_REPLY: nb("reply"), TAG_PRE: nb("pre_c1")}


class PartyProcess:
    """One party of the protocol.  run() is called by all three processes
    with the same parameters; P0 and P1 pass their own share, P2 passes
    None.  Returns the party's output share (None for P2)."""

    def __init__(self, party: int, stages: Stages, transport: Transport, clock=None):
        if party not in (P0, P1, P2):
            raise ValueError("party must be 0, 1 or 2")
        self.party = party
        self.s = stages
        self.tr = transport
        # optional: clock() -> seconds after the device finished its queued
        # work; with it, run() accumulates the party's own computing time
        # ("compute") and its time waiting for and moving messages ("transport")
        self.clock = clock
        self.timing = {"compute": 0.0, "transport": 0.0}

    def _lap(self, key: str, t0: float) -> float:
        if self.clock is None:
            return 0.0
        t = self.clock()
        self.timing[key] += t - t0
        return t

    def run(self, prm, relu: bool, share: Optional[torch.Tensor], n: int,
            tensor_id: int) -> Optional[torch.Tensor]:
        buf = self.s.buffers(prm, n)
        self.tr.prepare(self.party, message_sizes(buf))
        if self.party == P2:
            return self._helper(prm, relu, n, tensor_id, buf)
        return self._p01(prm, relu, share, n, tensor_id, buf)

    def _p01(self, prm, relu, share, n, tid, buf):
        me, other = self.party, 1 - self.party
        t = self.clock() if self.clock else 0.0
        w, opn = self.s.local(me, prm, relu, share, tid, buf)
        t = self._lap("compute", t)
        # round 1: w to P2; the openings between P0 and P1
        reqs = [self.tr.isend(w, me, P2, TAG_W)[0]]
        keep = []
        opens = [None, None]
        if relu:
            r, payload = self.tr.isend(opn, me, other, TAG_OPEN)
            reqs.append(r)
            keep.append(payload)
            rr, ob = self.tr.irecv(opn, other, TAG_OPEN)
            reqs.append(rr)
        # round 2: what P2 sends back
        rrep, rep = self.tr.irecv(buf["reply"], P2, TAG_REPLY) if (relu or me == P1) else (None,
                                                                                          None)
        rpre, pre = self.tr.irecv(buf["pre_c1"], P2, TAG_PRE) if (relu and me == P1) else (None,
                                                                                          None)
        wait_all([r for r in reqs + [rrep, rpre] if r is not None])
        if relu:
            opens[me], opens[other] = opn, self.tr.to_device(ob)
        reply = self.tr.to_device(rep) if rep is not None else None
        pre_c1 = self.tr.to_device(pre) if pre is not None else None
        t = self._lap("transport", t)
        out = self.s.finish(me, prm, relu, share, tid, reply, opens[0], opens[1], pre_c1, buf)
        self._lap("compute", t)
        return out

    def _helper(self, prm, relu, n, tid, buf):
        t = self.clock() if self.clock else 0.0
        r0, w0 = self.tr.irecv(buf["w"], P0, TAG_W)
        r1, w1 = self.tr.irecv(buf["w"], P1, TAG_W)
        wait_all([r0, r1])
        d0, d1 = self.tr.to_device(w0), self.tr.to_device(w1)
        t = self._lap("transport", t)
        reply, pre_c1 = self.s.helper(prm, relu, tid, d0, d1, buf)
        t = self._lap("compute", t)
        reqs, keep = [], []
        for dst, msg, tag in ([(P1, reply, TAG_REPLY)] if not relu else
                              [(P0, reply, TAG_REPLY), (P1, reply, TAG_REPLY),
                               (P1, pre_c1, TAG_PRE)]):
            r, payload = self.tr.isend(msg, P2, dst, tag)
            reqs.append(r)
            keep.append(payload)
        wait_all(reqs)
        self._lap("transport", t)
        return None
