"""Build and load the native library (libbicoptor.so, C-ABI in include/bicoptor.h).

The library is compiled in-tree with nvcc for sm_103a only.  There is no CPU
fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD, "libbicoptor.so")
SOURCES = ["bc_relu.cu", "bc_batch.cu", "bc_elementwise.cu", "bc_api.cu", "bc_noalloc.cu",
           "bc_parties.cu", "bc_peaks.cu", "bc_b1.cu"]
HEADERS = ["bc_device.cuh", "bc_element.cuh", "bc_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()
_lib = None


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbicoptor")


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "bicoptor.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit in parallel and link libbicoptor.so."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale():
        return LIB_PATH
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "--expt-relaxed-constexpr"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            print(err)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *[o for o, _ in results], "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ---- ctypes view of include/bicoptor.h -------------------------------------

c_int, c_u32, c_u64, c_size, c_void_p = (ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_size_t, ctypes.c_void_p)


class DreluParams(ctypes.Structure):
    _fields_ = [("ring_bits", c_int), ("lx", c_int), ("key_off", c_int), ("p", c_u32)]


class Comm(ctypes.Structure):
    _fields_ = [(n, c_u64) for n in ("p0_to_p2", "p1_to_p2", "p2_to_p0", "p2_to_p1", "p0_to_p1",
                                     "p1_to_p0", "pre_p2_to_p1", "rounds", "elements", "calls",
                                     "pre_p2_to_p0", "rss_reshare")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Audit(ctypes.Structure):
    _fields_ = [("w0", c_void_p), ("w1", c_void_p), ("reply", c_void_p), ("open0", c_void_p),
                ("open1", c_void_p), ("pre_c1", c_void_p), ("t", c_void_p), ("dprime", c_void_p)]


class TensorDesc(ctypes.Structure):
    _fields_ = [("sh0", c_void_p), ("sh1", c_void_p), ("o0", c_void_p), ("o1", c_void_p),
                ("n", c_u64), ("tensor_id", c_u32), ("op", c_int), ("params", DreluParams),
                ("elem_offset", c_u64)]


class PartyMsgs(ctypes.Structure):
    _fields_ = [("w0", c_void_p), ("w1", c_void_p), ("reply", c_void_p), ("open0", c_void_p),
                ("open1", c_void_p), ("pre_c1", c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("tile_elems", c_int), ("ctas_per_sm", c_int), ("schedule", c_int),
                ("elems_per_thread", c_int), ("slot_unroll", c_int)]


class IntPeaks(ctypes.Structure):
    _fields_ = [("imad_wide_per_s", ctypes.c_double), ("imad_per_s", ctypes.c_double),
                ("alu_per_s", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("sm_count", c_int), ("imad_hi_per_s", ctypes.c_double)]


class LinearReluArgs(ctypes.Structure):
    _fields_ = [("ring_bits", c_int), ("trunc_bits", c_int), ("relu", DreluParams),
                ("x0", c_void_p), ("x1", c_void_p), ("y0", c_void_p), ("y1", c_void_p),
                ("n", c_size), ("tensor_id", c_u32),
                ("prod0", c_void_p), ("prod1", c_void_p), ("trc0", c_void_p), ("trc1", c_void_p),
                ("det0", c_void_p), ("det1", c_void_p), ("relu0", c_void_p), ("relu1", c_void_p)]


P = ctypes.POINTER
SIGNATURES = {
    "bc_create": (c_int, [P(c_void_p), c_u64, c_int, c_void_p]),
    "bc_destroy": (c_int, [c_void_p]),
    "bc_set_stream": (c_int, [c_void_p, c_void_p]),
    "bc_synchronize": (c_int, [c_void_p]),
    "bc_strerror": (ctypes.c_char_p, [c_int]),
    "bc_last_cuda_error": (ctypes.c_char_p, [c_void_p]),
    "bc_prime_above": (c_u32, [c_int]),
    "bc_share": (c_int, [c_void_p, c_int, c_void_p, c_size, c_u32, c_void_p, c_void_p]),
    "bc_reconstruct": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_size, c_void_p]),
    "bc_trunc_prob": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_size, c_void_p,
                              c_void_p]),
    "bc_trunc_det": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_size, c_void_p,
                             c_void_p]),
    "bc_mod_switch": (c_int, [c_void_p, c_int, c_u32, c_void_p, c_void_p, c_size, c_void_p,
                              c_void_p]),
    "bc_mul_beaver": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_size,
                              c_u32, c_void_p, c_void_p]),
    "bc_drelu": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32, c_void_p,
                         c_void_p]),
    "bc_relu": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32, c_void_p,
                        c_void_p]),
    "bc_set_audit": (c_int, [c_void_p, P(Audit)]),
    "bc_get_comm": (c_int, [c_void_p, P(Comm)]),
    "bc_reset_comm": (c_int, [c_void_p]),
    "bc_drelu_b1": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32,
                            c_void_p, c_void_p, c_void_p, c_void_p]),
    "bc_relu_b1": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32,
                           c_void_p, c_void_p, c_void_p, c_void_p]),
    "bc_party_local": (c_int, [c_void_p, c_int, P(DreluParams), c_int, c_void_p, c_size, c_u32,
                               c_void_p, c_void_p]),
    "bc_party_helper": (c_int, [c_void_p, P(DreluParams), c_int, c_size, c_u32, c_void_p,
                                c_void_p, c_void_p, c_void_p]),
    "bc_party_finish": (c_int, [c_void_p, c_int, P(DreluParams), c_int, c_void_p, c_size, c_u32,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bc_relu_batch_plan": (c_int, [c_void_p, P(TensorDesc), c_int, P(BatchConfig)]),
    "bc_relu_batch_run": (c_int, [c_void_p]),
    "bc_relu_batch": (c_int, [c_void_p, P(TensorDesc), c_int, P(BatchConfig)]),
    "bc_relu_batch_host": (c_int, [c_void_p, P(TensorDesc), c_int, P(BatchConfig)]),
    "bc_batch_status": (c_int, [c_void_p]),
    "bc_linear_relu": (c_int, [c_void_p, P(LinearReluArgs)]),
    "bc_linear_relu_host": (c_int, [c_void_p, P(LinearReluArgs)]),
    "bc_reserve": (c_int, [c_void_p, c_size]),
    "bc_set_host_path": (c_int, [c_void_p, c_int]),
    "bc_set_checked": (c_int, [c_void_p, c_int]),
    "bc_measure_int_peaks": (c_int, [c_int, P(IntPeaks)]),
    "bc_count_trunc_failures": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                        c_size, c_void_p]),
    "bc_relu_batch_static": (c_int, [c_u64, c_int, c_void_p, P(TensorDesc), c_int, c_int]),
    "bc_relu_batch_static_status": (c_int, [c_int, c_void_p]),
    "bc_party_msg_words": (c_size, [c_int, c_size]),
    "bc_parties_status": (c_int, [c_void_p]),
    "bc_test_drop_p2_copies": (c_int, [c_void_p, c_int]),
    "bc_rss_drelu": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_void_p, c_size, c_u32,
                             c_void_p, c_void_p, c_void_p]),
    "bc_rss_relu": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_void_p, c_size, c_u32,
                            c_void_p, c_void_p, c_void_p]),
    "bc_trunc_aby3": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_size, c_u32, c_u64,
                              c_void_p, c_void_p]),
    "bc_trunc_then_mul": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_size, c_u32, c_void_p, c_void_p]),
    "bc_drelu_parties": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32,
                                 c_void_p, c_void_p, P(PartyMsgs)]),
    "bc_relu_parties": (c_int, [c_void_p, P(DreluParams), c_void_p, c_void_p, c_size, c_u32,
                                c_void_p, c_void_p, P(PartyMsgs)]),
}


def lib(build_if_missing: bool = True):
    """The loaded library; builds it first if needed.  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libbicoptor.so is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib
