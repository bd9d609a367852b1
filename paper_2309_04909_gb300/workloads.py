"""Seeded synthetic inputs for the Bicoptor 2.0 DReLU/ReLU workloads.

This module draws plaintext activations (as float64 reals) and the shapes of
the ReLU sets of the networks the paper evaluates (Sec. 6: AlexNet/VGG16-style
CNNs on CIFAR10 / Tiny ImageNet). It holds none of the protocol's arithmetic:
no fixed-point encoding, no sharing, no randomness that the protocol draws.
Both the CUDA path and the CPU oracle take their inputs from here.

The paper's datasets and trained weights are not available; these seeded
distributions stand in for the activations that reach a ReLU layer.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

# Per-image ReLU tensor sizes (channels * height * width) of the layers.
# VGG-16 on a 32x32x3 input: 13 ReLU layers after the 13 convolutions.
VGG16_32_LAYERS: List[int] = (
    [64 * 32 * 32] * 2 + [128 * 16 * 16] * 2 + [256 * 8 * 8] * 3
    + [512 * 4 * 4] * 3 + [512 * 2 * 2] * 3
)
# ResNet-18 on a 224x224x3 input: stem ReLU + 4 stages of 4 ReLUs.
RESNET18_224_LAYERS: List[int] = (
    [64 * 112 * 112] + [64 * 56 * 56] * 4 + [128 * 28 * 28] * 4
    + [256 * 14 * 14] * 4 + [512 * 7 * 7] * 4
)
# LeNet-style network on a 1x28x28 input: two conv ReLUs and two FC ReLUs.
LENET_28_LAYERS: List[int] = [6 * 24 * 24, 16 * 8 * 8, 120, 84]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_reals(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n reals uniform in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=n)


def gaussian_reals(n: int, sigma: float, seed: int, stream: int = 0) -> np.ndarray:
    """n reals from N(0, sigma^2); `stream` picks an independent sub-stream."""
    g = np.random.Generator(np.random.PCG64([seed, stream]))
    return g.normal(0.0, sigma, size=n)


def laplace_reals(n: int, scale: float, seed: int, stream: int = 0) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64([seed, stream]))
    return g.laplace(0.0, scale, size=n)


def magnitude_bounded_ints(n: int, bits: int, seed: int) -> np.ndarray:
    """Signed integers uniform in (-2^bits, 2^bits), as int64 (bits <= 62).

    Used directly as ring elements (already fixed-point), e.g. for the
    probabilistic-truncation failure sweep."""
    g = rng(seed)
    mag = g.integers(0, 1 << bits, size=n, dtype=np.int64)
    sign = g.integers(0, 2, size=n, dtype=np.int64)
    return np.where(sign == 1, -mag, mag)


@dataclasses.dataclass
class TensorSet:
    """A batch of ReLU input tensors: reals plus per-tensor metadata."""
    sizes: List[int]            # elements per tensor
    reals: List[np.ndarray]     # one float64 array per tensor
    ring_bits: List[int]
    frac_bits: List[int]
    name: str

    @property
    def total(self) -> int:
        return int(sum(self.sizes))


def vgg16_batch(batch: int, seed: int, layers=VGG16_32_LAYERS,
                ring_bits: int = 64, frac_bits: int = 16) -> TensorSet:
    """Per-image ReLU tensors of a VGG-16-shaped CNN; per-layer sigma drawn
    uniformly in [0.5, 8], values N(0, sigma^2)."""
    g = rng(seed)
    sigmas = g.uniform(0.5, 8.0, size=len(layers))
    sizes, reals = [], []
    for img in range(batch):
        for li, sz in enumerate(layers):
            sizes.append(sz)
            reals.append(gaussian_reals(sz, float(sigmas[li]), seed, stream=1 + img * 64 + li))
    nt = len(sizes)
    return TensorSet(sizes, reals, [ring_bits] * nt, [frac_bits] * nt, "vgg16-32x32")


def resnet18_mixed_batch(batch: int, seed: int, layers=RESNET18_224_LAYERS) -> TensorSet:
    """Per-image ReLU tensors of a ResNet-18-shaped CNN, once in Z_{2^64}
    (f=16) and once more in Z_{2^32} (f=12); Laplace(0, 2) activations."""
    sizes, reals, rb, fb = [], [], [], []
    for ring, frac, s in ((64, 16, 0), (32, 12, 1)):
        for img in range(batch):
            for li, sz in enumerate(layers):
                sizes.append(sz)
                reals.append(laplace_reals(sz, 2.0, seed, stream=1 + s * 100000 + img * 64 + li))
                rb.append(ring)
                fb.append(frac)
    return TensorSet(sizes, reals, rb, fb, "resnet18-224x224-mixed")


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    images: int
    net: str            # "lenet" or "vgg16"
    sizes: List[int]


def serving_trace(rate_per_s: float, duration_s: float, seed: int,
                  max_images: int = 64) -> List[Request]:
    """Poisson arrivals; each request is 1..max_images images of a LeNet- or
    VGG-16-shaped ReLU set (50/50)."""
    g = rng(seed)
    t, out, rid = 0.0, [], 0
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        images = int(g.integers(1, max_images + 1))
        net = "lenet" if g.integers(0, 2) == 0 else "vgg16"
        layers = LENET_28_LAYERS if net == "lenet" else VGG16_32_LAYERS
        out.append(Request(rid, t, images, net, [s for _ in range(images) for s in layers]))
        rid += 1
    return out


def request_reals(req: Request, seed: int) -> List[np.ndarray]:
    """Activations for one serving request (per-layer sigma in [0.5, 8])."""
    g = np.random.Generator(np.random.PCG64([seed, 7, req.rid]))
    nl = len(LENET_28_LAYERS if req.net == "lenet" else VGG16_32_LAYERS)
    sig = g.uniform(0.5, 8.0, size=nl)
    return [g.normal(0.0, float(sig[i % nl]), size=sz) for i, sz in enumerate(req.sizes)]
