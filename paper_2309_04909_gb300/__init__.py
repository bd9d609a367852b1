"""GB300-native Bicoptor 2.0 hot path: secret-shared truncation, modulo switch
and DReLU/ReLU over Z_{2^l} with three parties simulated on one GPU.

This module is a thin binding over the C-ABI of include/bicoptor.h: it
marshals torch tensors (device memory, streams) into plain pointers.  Every
step of the protocol runs in the CUDA kernels of libbicoptor.so; there is no
CPU fallback, and every call raises if the library is missing.

Lanes: a ring element of Z_{2^l} is stored in an int32 tensor (l <= 32) or an
int64 tensor (l <= 64), read as unsigned; Z_p values in int32 tensors.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Dict, Optional, Sequence, Tuple

import torch

from . import _native
from ._native import Audit, BatchConfig, Comm, DreluParams, LinearReluArgs, PartyMsgs, TensorDesc

__all__ = ["Context", "Params", "BicoptorError", "lane_dtype", "prime_above", "build"]

OP_RELU, OP_DRELU = 0, 1


class BicoptorError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    return _native.build(force=force)


def lane_dtype(bits: int) -> torch.dtype:
    return torch.int64 if bits > 32 else torch.int32


def prime_above(lx: int) -> int:
    return int(_native.lib().bc_prime_above(lx))


@dataclass(frozen=True)
class Params:
    """Alg. drelu parameters: ring bits l, key bits lx, key offset c, prime p (0 = derive)."""
    ring_bits: int
    lx: int
    key_off: int = 0
    p: int = 0

    def c_struct(self) -> DreluParams:
        # one ctypes struct per distinct parameter set (the library only reads it)
        c = _PRM_STRUCTS.get(self)
        if c is None:
            c = _PRM_STRUCTS[self] = DreluParams(self.ring_bits, self.lx, self.key_off, self.p)
        return c

    @property
    def slots(self) -> int:
        return self.lx + 1

    @classmethod
    def from_key_bits(cls, ring_bits: int, int_bits: int, frac_bits: int, kept_frac_bits: int,
                      p: int = 0) -> "Params":
        """The key bits of Sec. 6.1: the DReLU of a fixed-point value with
        int_bits integer and frac_bits fractional bits looks only at the integer
        bits and the top kept_frac_bits fractional bits.  So lx = int_bits +
        kept_frac_bits, and the lowest key bit is c = frac_bits - kept_frac_bits
        (l = 64 with 5 + 26 bits and 2 fractional bits kept gives lx = 7, c = 24:
        the last 24 bits ignored).  The windows of step 3 then need c + 2 lx <= l."""
        if not (0 <= kept_frac_bits <= frac_bits and int_bits >= 0):
            raise ValueError("need 0 <= kept_frac_bits <= frac_bits and int_bits >= 0")
        lx, c = int_bits + kept_frac_bits, frac_bits - kept_frac_bits
        if not 1 <= lx <= 31:
            raise ValueError(f"key bits lx = {lx} outside 1..31")
        if c + 2 * lx > ring_bits:
            raise ValueError(f"c + 2 lx = {c + 2 * lx} exceeds the ring's {ring_bits} bits")
        return cls(ring_bits, lx, c, p)


_PRM_STRUCTS: Dict["Params", DreluParams] = {}
# the current stream's raw cudaStream_t of a device, as an int (torch's own accessor)
_RAW_STREAM = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _ptr(t: Optional[torch.Tensor]):
    # a plain int: ctypes converts it for c_void_p arguments and fields
    return None if t is None else t.data_ptr()


class Context:
    """A simulation context: one device, one stream, one 64-bit seed from which
    every pre-shared seed (seed01, seed02, seed12, dealer) is keyed."""

    def __init__(self, seed: int, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self._lib = _native.lib()
        self.device = torch.device("cuda", device)
        self._dev_index = device
        self._stream = stream
        self._last_stream = None
        h = ctypes.c_void_p()
        self._check(self._lib.bc_create(ctypes.byref(h), seed, device, self._stream_handle()))
        self._h = h
        self.seed = seed

    # -- plumbing -------------------------------------------------------------
    def _stream_handle(self):
        s = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _sync_stream(self):
        # calls follow torch's current stream unless a stream was pinned; the
        # library is told only when the stream changes.  The raw handle is read
        # without building a Stream object where torch offers that.
        if self._stream is not None:
            h = self._stream.cuda_stream
        elif _RAW_STREAM is not None:
            h = _RAW_STREAM(self._dev_index)
        else:
            h = torch.cuda.current_stream(self.device).cuda_stream
        if h != self._last_stream:
            self._lib.bc_set_stream(self._h, h)
            self._last_stream = h

    def _check(self, rc: int):
        if rc != 0:
            msg = self._lib.bc_strerror(rc).decode()
            extra = ""
            if getattr(self, "_h", None) is not None:
                extra = self._lib.bc_last_cuda_error(self._h).decode()
            raise BicoptorError(f"bicoptor error {rc}: {msg} {extra}".strip())

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.bc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n: int, bits: int) -> torch.Tensor:
        return torch.empty(n, dtype=lane_dtype(bits), device=self.device)

    @staticmethod
    def _need(t: torch.Tensor, bits: int, name: str):
        if (t.dtype is not (torch.int64 if bits > 32 else torch.int32) or not t.is_cuda
                or not t.is_contiguous()):
            raise BicoptorError(f"{name}: expected a contiguous CUDA {lane_dtype(bits)} tensor")

    # -- sharing ----------------------------------------------------------------
    def share(self, ring_bits: int, x_fixed: torch.Tensor, tensor_id: int):
        if x_fixed.dtype != torch.int64 or not x_fixed.is_cuda:
            raise BicoptorError("share: x must be a CUDA int64 tensor of fixed-point values")
        x_fixed = x_fixed.contiguous()
        n = x_fixed.numel()
        s0, s1 = self._empty(n, ring_bits), self._empty(n, ring_bits)
        self._sync_stream()
        self._check(self._lib.bc_share(self._h, ring_bits, _ptr(x_fixed), n, tensor_id,
                                       _ptr(s0), _ptr(s1)))
        return s0, s1

    def reconstruct(self, ring_bits: int, s0: torch.Tensor, s1: torch.Tensor) -> torch.Tensor:
        self._need(s0, ring_bits, "s0")
        self._need(s1, ring_bits, "s1")
        out = self._empty(s0.numel(), ring_bits)
        self._sync_stream()
        self._check(self._lib.bc_reconstruct(self._h, ring_bits, _ptr(s0), _ptr(s1), s0.numel(),
                                             _ptr(out)))
        return out

    # -- truncations, modulo switch, product ------------------------------------
    def trunc_prob(self, ring_bits: int, k: int, s0, s1, out=None):
        self._need(s0, ring_bits, "s0")
        self._need(s1, ring_bits, "s1")
        n = s0.numel()
        o0, o1 = out if out is not None else (self._empty(n, ring_bits), self._empty(n, ring_bits))
        self._sync_stream()
        self._check(self._lib.bc_trunc_prob(self._h, ring_bits, k, _ptr(s0), _ptr(s1), n,
                                            _ptr(o0), _ptr(o1)))
        return o0, o1

    def trunc_det(self, ring_bits: int, k1: int, k2: int, s0, s1, out=None):
        self._need(s0, ring_bits, "s0")
        self._need(s1, ring_bits, "s1")
        n, ob = s0.numel(), ring_bits - k1 - k2
        o0, o1 = out if out is not None else (self._empty(n, ob), self._empty(n, ob))
        self._sync_stream()
        self._check(self._lib.bc_trunc_det(self._h, ring_bits, k1, k2, _ptr(s0), _ptr(s1), n,
                                           _ptr(o0), _ptr(o1)))
        return o0, o1

    def mod_switch(self, lp: int, p: int, s0, s1):
        self._need(s0, lp, "s0")
        self._need(s1, lp, "s1")
        n = s0.numel()
        o0 = torch.empty(n, dtype=torch.int32, device=self.device)
        o1 = torch.empty(n, dtype=torch.int32, device=self.device)
        self._sync_stream()
        self._check(self._lib.bc_mod_switch(self._h, lp, p, _ptr(s0), _ptr(s1), n, _ptr(o0),
                                            _ptr(o1)))
        return o0, o1

    def mul_beaver(self, ring_bits: int, x0, x1, y0, y1, tensor_id: int, out=None):
        for t, nm in ((x0, "x0"), (x1, "x1"), (y0, "y0"), (y1, "y1")):
            self._need(t, ring_bits, nm)
        n = x0.numel()
        o0, o1 = out if out is not None else (self._empty(n, ring_bits), self._empty(n, ring_bits))
        self._sync_stream()
        self._check(self._lib.bc_mul_beaver(self._h, ring_bits, _ptr(x0), _ptr(x1), _ptr(y0),
                                            _ptr(y1), n, tensor_id, _ptr(o0), _ptr(o1)))
        return o0, o1

    def trunc_aby3(self, ring_bits: int, k: int, s0, s1, tensor_id: int, fixed_r: int = 0,
                   out=None):
        """Alg. aby3trc; fixed_r != 0 uses the constant mask of Sec. 4.1."""
        self._need(s0, ring_bits, "s0")
        self._need(s1, ring_bits, "s1")
        n = s0.numel()
        o0, o1 = out if out is not None else (self._empty(n, ring_bits), self._empty(n, ring_bits))
        self._sync_stream()
        self._check(self._lib.bc_trunc_aby3(self._h, ring_bits, k, _ptr(s0), _ptr(s1), n,
                                            tensor_id, fixed_r, _ptr(o0), _ptr(o1)))
        return o0, o1

    def trunc_then_mul(self, ring_bits: int, kx: int, ky: int, x0, x1, y0, y1, tensor_id: int,
                       out=None):
        """Alg. linear: Alg. smltrc by kx / ky bits, then the Beaver product."""
        for t, nm in ((x0, "x0"), (x1, "x1"), (y0, "y0"), (y1, "y1")):
            self._need(t, ring_bits, nm)
        n = x0.numel()
        o0, o1 = out if out is not None else (self._empty(n, ring_bits), self._empty(n, ring_bits))
        self._sync_stream()
        self._check(self._lib.bc_trunc_then_mul(self._h, ring_bits, kx, ky, _ptr(x0), _ptr(x1),
                                                _ptr(y0), _ptr(y1), n, tensor_id, _ptr(o0),
                                                _ptr(o1)))
        return o0, o1

    # -- DReLU / ReLU -------------------------------------------------------------
    def _protocol(self, fn, prm: Params, s0, s1, tensor_id, out, audit):
        self._need(s0, prm.ring_bits, "s0")
        self._need(s1, prm.ring_bits, "s1")
        n = s0.numel()
        o0, o1 = out if out is not None else (self._empty(n, prm.ring_bits),
                                              self._empty(n, prm.ring_bits))
        bufs = None
        self._sync_stream()
        if audit:
            L = prm.slots
            dev = self.device
            bufs = dict(w0=torch.empty(n * L, dtype=torch.int32, device=dev),
                        w1=torch.empty(n * L, dtype=torch.int32, device=dev),
                        reply=self._empty(n, prm.ring_bits), open0=self._empty(n, prm.ring_bits),
                        open1=self._empty(n, prm.ring_bits), pre_c1=self._empty(n, prm.ring_bits),
                        t=torch.empty(n, dtype=torch.uint8, device=dev),
                        dprime=torch.empty(n, dtype=torch.uint8, device=dev))
            a = Audit(*[_ptr(bufs[k]) for k in ("w0", "w1", "reply", "open0", "open1", "pre_c1",
                                                 "t", "dprime")])
            self._check(self._lib.bc_set_audit(self._h, ctypes.byref(a)))
        try:
            prm_c = prm.c_struct()
            self._check(fn(self._h, ctypes.byref(prm_c), _ptr(s0), _ptr(s1), n, tensor_id,
                           _ptr(o0), _ptr(o1)))
        finally:
            if audit:
                self._lib.bc_set_audit(self._h, None)
        return (o0, o1, bufs) if audit else (o0, o1)

    def drelu(self, prm: Params, s0, s1, tensor_id: int, out=None, audit: bool = False):
        return self._protocol(self._lib.bc_drelu, prm, s0, s1, tensor_id, out, audit)

    def relu(self, prm: Params, s0, s1, tensor_id: int, out=None, audit: bool = False):
        return self._protocol(self._lib.bc_relu, prm, s0, s1, tensor_id, out, audit)

    # -- the Bicoptor 1.0-style baseline ---------------------------------------------
    def _b1(self, fn, prm: Params, s0, s1, tensor_id, out, messages):
        self._need(s0, prm.ring_bits, "s0")
        self._need(s1, prm.ring_bits, "s1")
        n = s0.numel()
        o0, o1 = out if out is not None else (self._empty(n, prm.ring_bits),
                                              self._empty(n, prm.ring_bits))
        w = None
        if messages:
            w = (self._empty(n * prm.slots, prm.ring_bits), self._empty(n * prm.slots,
                                                                          prm.ring_bits))
        self._sync_stream()
        self._check(fn(self._h, ctypes.byref(prm.c_struct()), _ptr(s0), _ptr(s1), n, tensor_id,
                       _ptr(o0), _ptr(o1), _ptr(w[0]) if w else None,
                       _ptr(w[1]) if w else None))
        return (o0, o1, w[0], w[1]) if messages else (o0, o1)

    def drelu_b1(self, prm: Params, s0, s1, tensor_id: int, out=None, messages: bool = False):
        """The Bicoptor 1.0-style DReLU (bc_drelu_b1): SecureML truncations,
        recursive sums and masks in Z_{2^l}; (lx+1) l bits per party.  With
        messages, also returns the two parties' messages to P2 (n * (lx+1))."""
        return self._b1(self._lib.bc_drelu_b1, prm, s0, s1, tensor_id, out, messages)

    def relu_b1(self, prm: Params, s0, s1, tensor_id: int, out=None, messages: bool = False):
        return self._b1(self._lib.bc_relu_b1, prm, s0, s1, tensor_id, out, messages)

    # -- RSS (Alg. drelu2) -----------------------------------------------------------
    def _rss(self, fn, prm: Params, x0, x1, x2, tensor_id, out):
        for t, nm in ((x0, "x0"), (x1, "x1"), (x2, "x2")):
            self._need(t, prm.ring_bits, nm)
        n = x0.numel()
        ys = out if out is not None else tuple(self._empty(n, prm.ring_bits) for _ in range(3))
        prm_c = prm.c_struct()
        self._sync_stream()
        self._check(fn(self._h, ctypes.byref(prm_c), _ptr(x0), _ptr(x1), _ptr(x2), n, tensor_id,
                       *[_ptr(y) for y in ys]))
        return ys

    def rss_drelu(self, prm: Params, x0, x1, x2, tensor_id: int, out=None):
        """Alg. drelu2 on replicated components; returns (y0, y1, y2)."""
        return self._rss(self._lib.bc_rss_drelu, prm, x0, x1, x2, tensor_id, out)

    def rss_relu(self, prm: Params, x0, x1, x2, tensor_id: int, out=None):
        return self._rss(self._lib.bc_rss_relu, prm, x0, x1, x2, tensor_id, out)

    # -- party-separated ----------------------------------------------------------
    def party_buffers(self, prm: Params, n: int) -> Dict[str, torch.Tensor]:
        """Message buffers of one party-separated call (see bc_party_msgs)."""
        words = int(self._lib.bc_party_msg_words(prm.lx, n))
        dev = self.device
        d = {"w0": torch.empty(words, dtype=torch.int32, device=dev),
             "w1": torch.empty(words, dtype=torch.int32, device=dev)}
        for k in ("reply", "open0", "open1", "pre_c1"):
            d[k] = self._empty(n, prm.ring_bits)
        return d

    def _parties(self, fn, prm: Params, s0, s1, tensor_id, out, msgs):
        self._need(s0, prm.ring_bits, "s0")
        self._need(s1, prm.ring_bits, "s1")
        n = s0.numel()
        o0, o1 = out if out is not None else (self._empty(n, prm.ring_bits),
                                              self._empty(n, prm.ring_bits))
        m = msgs if msgs is not None else self.party_buffers(prm, n)
        pm = PartyMsgs(*[_ptr(m[k]) for k in ("w0", "w1", "reply", "open0", "open1", "pre_c1")])
        prm_c = prm.c_struct()
        self._sync_stream()
        self._check(fn(self._h, ctypes.byref(prm_c), _ptr(s0), _ptr(s1), n, tensor_id, _ptr(o0),
                       _ptr(o1), ctypes.byref(pm)))
        return o0, o1, m

    def drelu_parties(self, prm: Params, s0, s1, tensor_id: int, out=None, msgs=None):
        """DReLU with each party's work in its own kernel and the messages in
        device buffers; returns (o0, o1, message buffers)."""
        return self._parties(self._lib.bc_drelu_parties, prm, s0, s1, tensor_id, out, msgs)

    def relu_parties(self, prm: Params, s0, s1, tensor_id: int, out=None, msgs=None):
        return self._parties(self._lib.bc_relu_parties, prm, s0, s1, tensor_id, out, msgs)

    # -- one party's stage (parties in separate processes; see parties.py) -------
    def party_stage_buffers(self, prm: Params, n: int) -> Dict[str, torch.Tensor]:
        """This party's buffers for one party-separated call: its packed w
        message ("w", also the size of a received one), its opening, the
        reply and [c]_1 it receives, and its output share."""
        words = int(self._lib.bc_party_msg_words(prm.lx, n))
        d = {"w": torch.empty(words, dtype=torch.int32, device=self.device)}
        for k in ("open", "reply", "pre_c1", "out"):
            d[k] = self._empty(n, prm.ring_bits)
        return d

    def party_local(self, party: int, prm: Params, relu: bool, share, tensor_id: int, buf):
        """bc_party_local: P0 (party 0) or P1 (party 1), steps 1-8 from its own
        share; returns (its packed w message, its opening or None)."""
        self._need(share, prm.ring_bits, "share")
        w, opn = buf["w"], (buf["open"] if relu else None)
        self._sync_stream()
        self._check(self._lib.bc_party_local(self._h, party, ctypes.byref(prm.c_struct()),
                                             int(relu), _ptr(share), share.numel(), tensor_id,
                                             _ptr(w), _ptr(opn)))
        return w, opn

    def party_helper(self, prm: Params, relu: bool, tensor_id: int, w0, w1, buf):
        """bc_party_helper: P2's step 9 on the two received w messages;
        returns (reply, [c]_1 or None)."""
        n = buf["reply"].numel()
        reply, pre = buf["reply"], (buf["pre_c1"] if relu else None)
        self._sync_stream()
        self._check(self._lib.bc_party_helper(self._h, ctypes.byref(prm.c_struct()), int(relu), n,
                                              tensor_id, _ptr(w0), _ptr(w1), _ptr(reply),
                                              _ptr(pre)))
        return reply, pre

    def party_finish(self, party: int, prm: Params, relu: bool, share, tensor_id: int, reply,
                     open0, open1, pre_c1, buf):
        """bc_party_finish: P0 or P1 finishes from the messages it received;
        returns its output share."""
        out = buf["out"]
        self._sync_stream()
        self._check(self._lib.bc_party_finish(self._h, party, ctypes.byref(prm.c_struct()),
                                              int(relu), _ptr(share), out.numel(), tensor_id,
                                              _ptr(reply), _ptr(open0), _ptr(open1),
                                              _ptr(pre_c1), _ptr(out)))
        return out

    def parties_status(self) -> int:
        """0, or BC_ETIMEOUT (-4) if P2's bounded wait for its messages gave up
        in a party-separated call since the last read; synchronises, clears."""
        return int(self._lib.bc_parties_status(self._h))

    def test_drop_p2_copies(self, on: bool = True):
        """Test hook: P2's kernel issues no message copies, so its wait runs out."""
        self._check(self._lib.bc_test_drop_p2_copies(self._h, 1 if on else 0))

    # -- batched ------------------------------------------------------------------
    def relu_batch_plan(self, items: Sequence[Tuple], tile_elems: int = 0, ctas_per_sm: int = 0,
                        schedule: int = 0, elems_per_thread: int = 0, slot_unroll: int = 0):
        """items: (prm, s0, s1, o0, o1, tensor_id[, op[, elem_offset]]) per tensor;
        schedule 0 = persistent tile queue, 1 = one CTA per tile of 256 x
        elems_per_thread elements; slot_unroll = unroll of the key-bit loop
        (0 = default)."""
        arr = (TensorDesc * max(1, len(items)))()
        self._batch_keep = list(items)
        for i, it in enumerate(items):
            prm, s0, s1, o0, o1, tid = it[:6]
            op = it[6] if len(it) > 6 else OP_RELU
            off = it[7] if len(it) > 7 else 0
            for t, nm in ((s0, "s0"), (s1, "s1"), (o0, "o0"), (o1, "o1")):
                self._need(t, prm.ring_bits, nm)
            arr[i] = TensorDesc(s0.data_ptr(), s1.data_ptr(), o0.data_ptr(), o1.data_ptr(),
                                s0.numel(), tid, op, prm.c_struct(), off)
        cfg = BatchConfig(tile_elems, ctas_per_sm, schedule, elems_per_thread, slot_unroll)
        self._sync_stream()
        self._check(self._lib.bc_relu_batch_plan(self._h, arr, len(items), ctypes.byref(cfg)))

    def relu_batch_plan_descs(self, descs, count: int, tile_elems: int = 0, ctas_per_sm: int = 0,
                              schedule: int = 0, elems_per_thread: int = 0, slot_unroll: int = 0):
        """Plan from a prepared ctypes array of TensorDesc (raw device
        pointers; the caller keeps the memory alive)."""
        cfg = BatchConfig(tile_elems, ctas_per_sm, schedule, elems_per_thread, slot_unroll)
        self._sync_stream()
        self._check(self._lib.bc_relu_batch_plan(self._h, descs, count, ctypes.byref(cfg)))

    def relu_batch_host(self, items: Sequence[Tuple], tile_elems: int = 0, ctas_per_sm: int = 0,
                        schedule: int = 0, elems_per_thread: int = 0, slot_unroll: int = 0):
        """The batched DReLU/ReLU on pinned HOST tensors (bc_relu_batch_host):
        items as for relu_batch_plan, with page-locked CPU tensors (e.g.
        pin_memory()); the kernel reads and writes them across the host link.
        Returns once the outputs are in host memory."""
        arr = (TensorDesc * max(1, len(items)))()
        for i, it in enumerate(items):
            prm, s0, s1, o0, o1, tid = it[:6]
            op = it[6] if len(it) > 6 else OP_RELU
            off = it[7] if len(it) > 7 else 0
            for t, nm in ((s0, "s0"), (s1, "s1"), (o0, "o0"), (o1, "o1")):
                if (t.dtype is not lane_dtype(prm.ring_bits) or t.is_cuda or not t.is_contiguous()
                        or (t.numel() and not t.is_pinned())):
                    raise BicoptorError(f"{nm}: expected a contiguous pinned CPU "
                                        f"{lane_dtype(prm.ring_bits)} tensor")
            arr[i] = TensorDesc(s0.data_ptr(), s1.data_ptr(), o0.data_ptr(), o1.data_ptr(),
                                s0.numel(), tid, op, prm.c_struct(), off)
        cfg = BatchConfig(tile_elems, ctas_per_sm, schedule, elems_per_thread, slot_unroll)
        self._sync_stream()
        self._check(self._lib.bc_relu_batch_host(self._h, arr, len(items), ctypes.byref(cfg)))

    @staticmethod
    def batch_descs(items: Sequence[Tuple]):
        """A prepared ctypes array of bc_tensor_desc for `items` (tuples as for
        relu_batch_plan; device or pinned host tensors).  It records the
        buffers' addresses and sizes only, so it stays valid while the tensors
        live and may be passed to relu_batch_plan_descs / relu_batch_host_descs
        call after call.  Returns (array, count)."""
        arr = (TensorDesc * max(1, len(items)))()
        for i, it in enumerate(items):
            prm, s0, s1, o0, o1, tid = it[:6]
            op = it[6] if len(it) > 6 else OP_RELU
            off = it[7] if len(it) > 7 else 0
            arr[i] = TensorDesc(s0.data_ptr(), s1.data_ptr(), o0.data_ptr(), o1.data_ptr(),
                                s0.numel(), tid, op, prm.c_struct(), off)
        return arr, len(items)

    def relu_batch_host_descs(self, descs, count: int, tile_elems: int = 0, ctas_per_sm: int = 0,
                              schedule: int = 0, elems_per_thread: int = 0,
                              slot_unroll: int = 0):
        """bc_relu_batch_host on a prepared descriptor array (batch_descs) of
        pinned host buffers; the library checks that every buffer is mapped
        page-locked memory.  Returns once the outputs are in host memory."""
        cfg = BatchConfig(tile_elems, ctas_per_sm, schedule, elems_per_thread, slot_unroll)
        self._sync_stream()
        self._check(self._lib.bc_relu_batch_host(self._h, descs, count, ctypes.byref(cfg)))

    def relu_batch_run(self):
        self._sync_stream()
        self._check(self._lib.bc_relu_batch_run(self._h))

    def batch_status(self) -> int:
        return int(self._lib.bc_batch_status(self._h))

    # -- product -> truncations -> ReLU -------------------------------------------
    def linear_relu(self, ring_bits: int, k: int, prm: Params, x0, x1, y0, y1, tensor_id: int,
                    work=None):
        """Beaver product, Alg. smltrc and Alg. newtrc by k bits, ReLU of the
        probabilistically truncated product, in one fused kernel.  `work` maps
        output names to device tensors; "relu0"/"relu1" are required, the pairs
        "prod", "trc" and "det" are written only when present.  Returns `work`
        (all eight outputs when it is None)."""
        n = x0.numel()
        w = work or self.linear_relu_buffers(ring_bits, k, n)
        ptr = lambda nm: w[nm].data_ptr() if nm in w else None
        a = LinearReluArgs(ring_bits, k, prm.c_struct(), x0.data_ptr(), x1.data_ptr(),
                           y0.data_ptr(), y1.data_ptr(), n, tensor_id,
                           *[ptr(nm) for nm in ("prod0", "prod1", "trc0", "trc1", "det0",
                                                "det1", "relu0", "relu1")])
        self._sync_stream()
        self._check(self._lib.bc_linear_relu(self._h, ctypes.byref(a)))
        return w

    def linear_relu_buffers(self, ring_bits: int, k: int, n: int,
                            names=("prod0", "prod1", "trc0", "trc1", "det0", "det1", "relu0",
                                   "relu1")) -> Dict[str, torch.Tensor]:
        return {nm: self._empty(n, ring_bits - k if nm.startswith("det") else ring_bits)
                for nm in names}

    def set_checked(self, on: bool = True):
        """Checked mode: calls verify that their input lanes are canonical
        (no bits at or above l) and raise instead of running if not; each
        checked call waits for its check."""
        self._check(self._lib.bc_set_checked(self._h, 1 if on else 0))

    HOST_AUTO, HOST_DIRECT, HOST_STAGED = 0, 1, 2

    def set_host_path(self, path: int):
        """Path of linear_relu_host: HOST_AUTO (direct when every buffer is
        pinned), HOST_DIRECT, HOST_STAGED."""
        self._check(self._lib.bc_set_host_path(self._h, path))

    def reserve(self, max_chunk: int):
        self._check(self._lib.bc_reserve(self._h, max_chunk))

    def linear_relu_host(self, ring_bits: int, k: int, prm: Params, x0, x1, y0, y1,
                         tensor_id: int, out: Dict[str, torch.Tensor]):
        """Host tensors in and out ("relu0"/"relu1" required, "det0"/"det1"
        optional).  Pinned tensors take the direct path (the kernel reads and
        writes them across the host link); others are staged in chunks, which
        needs reserve() first."""
        n = x0.numel()
        det = [out[nm].data_ptr() if nm in out else None for nm in ("det0", "det1")]
        a = LinearReluArgs(ring_bits, k, prm.c_struct(), x0.data_ptr(), x1.data_ptr(),
                           y0.data_ptr(), y1.data_ptr(), n, tensor_id, None, None, None, None,
                           *det, out["relu0"].data_ptr(), out["relu1"].data_ptr())
        self._sync_stream()
        self._check(self._lib.bc_linear_relu_host(self._h, ctypes.byref(a)))
        return out

    # -- evaluation ---------------------------------------------------------------
    def count_trunc_failures(self, out_bits: int, k: int, x: torch.Tensor, o0, o1) -> int:
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._sync_stream()
        self._check(self._lib.bc_count_trunc_failures(self._h, out_bits, k, _ptr(x), _ptr(o0),
                                                      _ptr(o1), o0.numel(), _ptr(cnt)))
        return int(cnt.item())

    def comm(self) -> Dict[str, int]:
        c = Comm()
        self._check(self._lib.bc_get_comm(self._h, ctypes.byref(c)))
        return c.as_dict()

    def reset_comm(self):
        self._check(self._lib.bc_reset_comm(self._h))

    def synchronize(self):
        self._check(self._lib.bc_synchronize(self._h))


def measure_int_peaks(device: int = 0) -> Dict[str, float]:
    """Measured rates of the integer instructions that bound the hot path
    (bc_measure_int_peaks): widening products, 32-bit multiply-adds, high
    halves of products and integer-ALU instructions per second, with the SM
    clock seen during the runs."""
    lib = _native.lib()
    p = _native.IntPeaks()
    rc = lib.bc_measure_int_peaks(device, ctypes.byref(p))
    if rc != 0:
        raise BicoptorError(f"bc_measure_int_peaks failed: {lib.bc_strerror(rc).decode()}")
    return {"imad_wide_per_s": p.imad_wide_per_s, "imad_per_s": p.imad_per_s,
            "imad_hi_per_s": p.imad_hi_per_s, "alu_per_s": p.alu_per_s, "sm_mhz": p.sm_mhz,
            "sm_count": p.sm_count}


def relu_batch_static(seed: int, items: Sequence[Tuple], tile_elems: int = 0,
                      device: int = 0, stream: Optional[torch.cuda.Stream] = None) -> None:
    """Batched ReLU/DReLU through bc_relu_batch_static: for callers that may
    not allocate device memory (no Context needed; the library's fixed device
    scratch is used).  items as for Context.relu_batch_plan.  Raises on an
    error code; -6 (BC_ELIMIT) means the batch exceeds the fixed capacity of
    256 tensors / 16384 tiles."""
    lib = _native.lib()
    arr = (TensorDesc * max(1, len(items)))()
    for i, it in enumerate(items):
        prm, s0, s1, o0, o1, tid = it[:6]
        op = it[6] if len(it) > 6 else OP_RELU
        arr[i] = TensorDesc(s0.data_ptr(), s1.data_ptr(), o0.data_ptr(), o1.data_ptr(),
                            s0.numel(), tid, op, prm.c_struct(), it[7] if len(it) > 7 else 0)
    s = stream if stream is not None else torch.cuda.current_stream(device)
    rc = lib.bc_relu_batch_static(seed, device, ctypes.c_void_p(s.cuda_stream), arr, len(items),
                                  tile_elems)
    if rc == -6:
        raise BicoptorError("bc_relu_batch_static: batch exceeds the fixed scratch capacity "
                            "(256 tensors, 16384 tiles, 32 parameter groups)")
    if rc != 0:
        raise BicoptorError(f"bc_relu_batch_static failed: {lib.bc_strerror(rc).decode()}")


def relu_batch_static_status(device: int = 0, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Status word of the last relu_batch_static launch on `device` (0, or -5
    = BC_ECHECK for a skipped malformed tile); read and cleared in stream
    order, then the stream is synchronised."""
    lib = _native.lib()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(lib.bc_relu_batch_static_status(device, ctypes.c_void_p(s.cuda_stream)))


def to_unsigned_numpy(t: torch.Tensor):
    """Copy a lane tensor to host as a uint32/uint64 numpy array."""
    import numpy as np
    a = t.detach().cpu().numpy()
    return a.view(np.uint64 if a.dtype == np.int64 else np.uint32 if a.dtype == np.int32 else a.dtype)


def from_unsigned_numpy(a, device) -> torch.Tensor:
    import numpy as np
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a.copy()).to(device)
