"""Python view of the plain C oracle (oracle/bicoptor_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may import this package; the product path never does.  It shares no
code with the CUDA sources.

Every function takes and returns numpy arrays: ring elements as uint64 (any
l <= 64, reduced mod 2^l), Z_p values as uint32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BICOPTOR_ORACLE_SRC points the oracle at another copy of its source (the
# mutation tests build planted-mistake copies this way); the library of such a
# copy is built beside it, never over the real one.
_SRC = os.environ.get("BICOPTOR_ORACLE_SRC") or os.path.join(_HERE, "bicoptor_oracle.c")
_LIB_PATH = (os.path.join(os.path.dirname(os.path.abspath(_SRC)), "_build", "liboracle.so")
             if os.environ.get("BICOPTOR_ORACLE_SRC") else os.path.join(_HERE, "_build", "liboracle.so"))
_lock = threading.Lock()
_lib = None

PAIR_01, PAIR_02, PAIR_12, PAIR_DEALER, PAIR_012, PAIR_2 = 0x01, 0x02, 0x12, 0xDE, 0x03, 0x20
PUR_SHARE, PUR_PERM, PUR_MASK, PUR_REPLY, PUR_RELU_TRIPLE, PUR_MUL_TRIPLE, PUR_ABY3 = (
    1, 2, 3, 4, 5, 6, 7)
PUR_RSS_T, PUR_RSS_S, PUR_RSS_Z, PUR_RSS_ZR = 8, 9, 10, 11
PUR_B1_MASK = 12


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wextra",
           "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int), ("lx", ctypes.c_int), ("c", ctypes.c_int),
                ("p", ctypes.c_uint32)]


class _Audit(ctypes.Structure):
    _fields_ = [("w0", ctypes.c_void_p), ("w1", ctypes.c_void_p), ("reply", ctypes.c_void_p),
                ("open0", ctypes.c_void_p), ("open1", ctypes.c_void_p),
                ("pre_c1", ctypes.c_void_p), ("t", ctypes.c_void_p), ("dprime", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            u64 = ctypes.c_uint64
            _lib.orc_cut.restype = u64
            _lib.orc_cut.argtypes = [u64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            _lib.orc_prime_above.restype = ctypes.c_uint32
            _lib.orc_prime_above.argtypes = [ctypes.c_int]
            _lib.orc_stream_word.restype = ctypes.c_uint32
            _lib.orc_stream_word.argtypes = [u64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                                             u64, u64]
            _lib.orc_drelu_core.restype = ctypes.c_int
            _lib.orc_max_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _u64(a):
    return np.ascontiguousarray(np.asarray(a).astype(np.uint64, copy=False))


def ring_mask(ell: int) -> int:
    return (1 << ell) - 1


def prime_above(lx: int) -> int:
    return int(lib().orc_prime_above(lx))


def cut(alpha: int, ell: int, k1: int, k2: int = 0) -> int:
    return int(lib().orc_cut(alpha, ell, k1, k2))


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def stream_word(seed, pair, purpose, tid, elem, j) -> int:
    return int(lib().orc_stream_word(seed, pair, purpose, tid, elem, j))


def encode(x: np.ndarray, frac_bits: int, ell: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.shape, dtype=np.uint64)
    lib().orc_encode(_p(x), ctypes.c_size_t(x.size), frac_bits, ell, _p(out))
    return out


def to_signed(v: np.ndarray, ell: int) -> np.ndarray:
    v = _u64(v)
    out = np.empty(v.shape, dtype=np.int64)
    lib().orc_to_signed(_p(v), ctypes.c_size_t(v.size), ell, _p(out))
    return out


def share_with_r(ell: int, x: int, r: int):
    s0, s1 = ctypes.c_uint64(), ctypes.c_uint64()
    lib().orc_share_with_r(ell, ctypes.c_uint64(x), ctypes.c_uint64(r), ctypes.byref(s0),
                           ctypes.byref(s1))
    return s0.value, s1.value


def share(ell, x, seed, tid, idx=None):
    x = _u64(x)
    idx = None if idx is None else _u64(idx)
    s0 = np.empty_like(x)
    s1 = np.empty_like(x)
    lib().orc_share(ell, _p(x), _p(idx), ctypes.c_size_t(x.size), ctypes.c_uint64(seed),
                    ctypes.c_uint32(tid), _p(s0), _p(s1))
    return s0, s1


def reconstruct(ell, s0, s1):
    s0, s1 = _u64(s0), _u64(s1)
    out = np.empty_like(s0)
    lib().orc_reconstruct(ell, _p(s0), _p(s1), ctypes.c_size_t(s0.size), _p(out))
    return out


def trunc_prob(ell, k, s0, s1):
    s0, s1 = _u64(s0), _u64(s1)
    o0, o1 = np.empty_like(s0), np.empty_like(s1)
    lib().orc_trunc_prob(ell, k, _p(s0), _p(s1), ctypes.c_size_t(s0.size), _p(o0), _p(o1))
    return o0, o1


def trunc_det(ell, k1, k2, s0, s1):
    s0, s1 = _u64(s0), _u64(s1)
    o0, o1 = np.empty_like(s0), np.empty_like(s1)
    lib().orc_trunc_det(ell, k1, k2, _p(s0), _p(s1), ctypes.c_size_t(s0.size), _p(o0), _p(o1))
    return o0, o1


def mod_switch(lp, p, s0, s1):
    s0, s1 = _u64(s0), _u64(s1)
    o0 = np.empty(s0.shape, dtype=np.uint32)
    o1 = np.empty(s1.shape, dtype=np.uint32)
    lib().orc_mod_switch(lp, ctypes.c_uint32(p), _p(s0), _p(s1), ctypes.c_size_t(s0.size),
                         _p(o0), _p(o1))
    return o0, o1


def mul_beaver(ell, x0, x1, y0, y1, seed, tid, idx=None):
    x0, x1, y0, y1 = map(_u64, (x0, x1, y0, y1))
    idx = None if idx is None else _u64(idx)
    o0, o1 = np.empty_like(x0), np.empty_like(x0)
    lib().orc_mul_beaver(ell, _p(x0), _p(x1), _p(y0), _p(y1), _p(idx), ctypes.c_size_t(x0.size),
                         ctypes.c_uint64(seed), ctypes.c_uint32(tid), _p(o0), _p(o1))
    return o0, o1


def params(ell, lx, c=0, p=None):
    return _Params(ell, lx, c, prime_above(lx) if p is None else p)


def drelu_core(P: _Params, s0: int, s1: int, t: int, fy, r, z):
    """Steps 1-9 of Alg. drelu for one element with explicit randomness.
    Returns (DReLU', msg0, msg1)."""
    L = P.lx + 1
    fy_a = (ctypes.c_uint32 * L)(*([0] + list(fy)))   # fy[1..lx]
    r_a = (ctypes.c_uint32 * L)(*r)
    z_a = (ctypes.c_uint32 * L)(*z)
    m0 = (ctypes.c_uint32 * L)()
    m1 = (ctypes.c_uint32 * L)()
    d = lib().orc_drelu_core(ctypes.byref(P), ctypes.c_uint64(s0), ctypes.c_uint64(s1), t,
                             fy_a, r_a, z_a, m0, m1)
    return d, list(m0), list(m1)


def _run(fn, P, s0, s1, seed, tid, idx, audit, threads):
    s0, s1 = _u64(s0), _u64(s1)
    n = s0.size
    idx = None if idx is None else _u64(idx)
    o0, o1 = np.empty_like(s0), np.empty_like(s1)
    L = P.lx + 1
    aud = None
    bufs = {}
    if audit:
        bufs = dict(w0=np.empty((n, L), np.uint32), w1=np.empty((n, L), np.uint32),
                    reply=np.empty(n, np.uint64), open0=np.zeros(n, np.uint64),
                    open1=np.zeros(n, np.uint64), pre_c1=np.zeros(n, np.uint64),
                    t=np.empty(n, np.uint8), dprime=np.empty(n, np.uint8))
        aud = _Audit(*[_p(bufs[k]) for k in ("w0", "w1", "reply", "open0", "open1", "pre_c1",
                                              "t", "dprime")])
    rc = fn(ctypes.byref(P), _p(s0), _p(s1), _p(idx), ctypes.c_size_t(n), ctypes.c_uint64(seed),
            ctypes.c_uint32(tid), _p(o0), _p(o1), ctypes.byref(aud) if aud else None, threads)
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return (o0, o1, bufs) if audit else (o0, o1)


def drelu(P, s0, s1, seed, tid, idx=None, audit=False, threads=1):
    return _run(lib().orc_drelu, P, s0, s1, seed, tid, idx, audit, threads)


def relu(P, s0, s1, seed, tid, idx=None, audit=False, threads=1):
    return _run(lib().orc_relu, P, s0, s1, seed, tid, idx, audit, threads)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of the elementwise loops (sharing, truncations, modulo switch,
    products, reconstruct); 0 = all cores (OpenMP's default), 1 = one core.
    drelu, relu and rss_drelu take their own `threads` argument."""
    lib().orc_set_threads(int(n))


def drelu_core_many(P: _Params, s0, s1, t, fy, r, z):
    """Vectorised drelu_core: fy, r, z are (n, lx+1) uint32 arrays (fy[:, 0]
    unused).  Returns DReLU' per row."""
    s0, s1 = _u64(s0), _u64(s1)
    n = s0.size
    t = np.ascontiguousarray(t, dtype=np.uint8)
    fy, r, z = (np.ascontiguousarray(a, dtype=np.uint32) for a in (fy, r, z))
    out = np.empty(n, np.uint8)
    rc = lib().orc_drelu_core_many(ctypes.byref(P), _p(s0), _p(s1), _p(t), _p(fy), _p(r), _p(z),
                                   ctypes.c_size_t(n), _p(out))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return out


def aby3_core(ell, k, s0, s1, r0, r1, rp0):
    """One element of Alg. aby3trc with explicit preprocessing randomness."""
    o0, o1 = ctypes.c_uint64(), ctypes.c_uint64()
    u = ctypes.c_uint64
    lib().orc_aby3_core(ell, k, u(s0), u(s1), u(r0), u(r1), u(rp0), ctypes.byref(o0),
                        ctypes.byref(o1))
    return o0.value, o1.value


def trunc_aby3(ell, k, s0, s1, seed, tid, fixed_r=0, idx=None):
    s0, s1 = _u64(s0), _u64(s1)
    idx = None if idx is None else _u64(idx)
    o0, o1 = np.empty_like(s0), np.empty_like(s1)
    lib().orc_trunc_aby3(ell, k, _p(s0), _p(s1), _p(idx), ctypes.c_size_t(s0.size),
                         ctypes.c_uint64(seed), ctypes.c_uint32(tid), ctypes.c_uint64(fixed_r),
                         _p(o0), _p(o1))
    return o0, o1


def trunc_then_mul(ell, kx, ky, x0, x1, y0, y1, seed, tid, idx=None):
    x0, x1, y0, y1 = map(_u64, (x0, x1, y0, y1))
    idx = None if idx is None else _u64(idx)
    o0, o1 = np.empty_like(x0), np.empty_like(x0)
    lib().orc_trunc_then_mul(ell, kx, ky, _p(x0), _p(x1), _p(y0), _p(y1), _p(idx),
                             ctypes.c_size_t(x0.size), ctypes.c_uint64(seed),
                             ctypes.c_uint32(tid), _p(o0), _p(o1))
    return o0, o1


def rss_drelu(P, x0, x1, x2, seed, tid, relu=False, idx=None, threads=1):
    """Alg. drelu2 (relu=False) or the RSS ReLU on replicated components;
    returns (y0, y1, y2, DReLU')."""
    x0, x1, x2 = map(_u64, (x0, x1, x2))
    n = x0.size
    idx = None if idx is None else _u64(idx)
    y0, y1, y2 = (np.empty_like(x0) for _ in range(3))
    dp = np.empty(n, np.uint8)
    rc = lib().orc_rss_drelu(ctypes.byref(P), _p(x0), _p(x1), _p(x2), _p(idx), ctypes.c_size_t(n),
                             ctypes.c_uint64(seed), ctypes.c_uint32(tid), int(relu), _p(y0),
                             _p(y1), _p(y2), _p(dp), threads)
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return y0, y1, y2, dp


def b1(P, s0, s1, seed, tid, relu=False, idx=None, msgs=False, threads=1):
    """The Bicoptor 1.0-style DReLU (relu=False) or ReLU: SecureML truncations
    in Z_{2^l}, recursive sums, masking by odd units and the zero test in
    Z_{2^l}.  Returns (o0, o1) or, with msgs, (o0, o1, w0, w1, dprime) where
    w0/w1 are (n, lx+1) ring elements."""
    s0, s1 = _u64(s0), _u64(s1)
    n = s0.size
    idx = None if idx is None else _u64(idx)
    o0, o1 = np.empty_like(s0), np.empty_like(s1)
    L = P.lx + 1
    w0 = np.empty((n, L), np.uint64) if msgs else None
    w1 = np.empty((n, L), np.uint64) if msgs else None
    dp = np.empty(n, np.uint8) if msgs else None
    rc = lib().orc_b1(ctypes.byref(P), int(relu), _p(s0), _p(s1), _p(idx), ctypes.c_size_t(n),
                      ctypes.c_uint64(seed), ctypes.c_uint32(tid), _p(o0), _p(o1), _p(w0), _p(w1),
                      _p(dp), threads)
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return (o0, o1, w0, w1, dp) if msgs else (o0, o1)


def drelu_b1_core_many(P: _Params, s0, s1, t, fy, r, z):
    """Steps 1-9 of the 1.0-style protocol with explicit randomness: fy
    (n, lx+1) uint32 (fy[:, 0] unused), r and z (n, lx+1) ring elements (r
    odd).  Returns DReLU' per row."""
    s0, s1 = _u64(s0), _u64(s1)
    n = s0.size
    t = np.ascontiguousarray(t, dtype=np.uint8)
    fy = np.ascontiguousarray(fy, dtype=np.uint32)
    r, z = _u64(r), _u64(z)
    out = np.empty(n, np.uint8)
    rc = lib().orc_drelu_b1_core_many(ctypes.byref(P), _p(s0), _p(s1), _p(t), _p(fy), _p(r),
                                      _p(z), ctypes.c_size_t(n), _p(out))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return out
