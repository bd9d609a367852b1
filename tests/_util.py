"""Shared helpers of the test-suite (no protocol arithmetic here)."""
import numpy as np
import torch


def cuda_ok() -> bool:
    return torch.cuda.is_available()


def to_np(t: torch.Tensor) -> np.ndarray:
    a = t.detach().cpu().numpy()
    if a.dtype == np.int64:
        return a.view(np.uint64)
    if a.dtype == np.int32:
        return a.view(np.uint32)
    return a


def to_dev(a: np.ndarray, bits: int, device="cuda") -> torch.Tensor:
    a = np.ascontiguousarray(a).astype(np.uint64 if bits > 32 else np.uint32)
    return torch.from_numpy(a.view(np.int64 if bits > 32 else np.int32).copy()).to(device)


def encode_np(reals: np.ndarray, frac_bits: int) -> np.ndarray:
    """Fixed-point plaintexts as the data owner hands them to the dealer
    (round half to even), int64."""
    return np.rint(np.ldexp(reals, frac_bits)).astype(np.int64)


def masked(x_int: np.ndarray, bits: int) -> np.ndarray:
    m = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    return x_int.astype(np.uint64) & m
