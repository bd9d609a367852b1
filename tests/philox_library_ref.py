"""Philox-4x32-10 outputs from an independent library implementation.

Run as a script with TRITON_INTERPRET=1 so that Triton's own Philox
(triton.language.random.philox, a third-party implementation of the same
published generator) executes with numpy on the CPU.  Reads a JSON list of
[c0, c1, c2, c3, k0, k1] rows on stdin and prints the four output words of
each row as JSON.  Used only by the oracle's Philox pin.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_rows(inp, out, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(inp + i * 6 + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(inp + i * 6 + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(inp + i * 6 + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(inp + i * 6 + 3).to(tl.uint32, bitcast=True)
    k0 = tl.load(inp + i * 6 + 4).to(tl.uint32, bitcast=True)
    k1 = tl.load(inp + i * 6 + 5).to(tl.uint32, bitcast=True)
    o0, o1, o2, o3 = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out + i * 4 + 0, o0.to(tl.int32, bitcast=True))
    tl.store(out + i * 4 + 1, o1.to(tl.int32, bitcast=True))
    tl.store(out + i * 4 + 2, o2.to(tl.int32, bitcast=True))
    tl.store(out + i * 4 + 3, o3.to(tl.int32, bitcast=True))


def main():
    rows = json.load(sys.stdin)
    n = len(rows)
    N = 1
    while N < n:
        N *= 2
    arr = np.zeros((N, 6), dtype=np.uint32)
    arr[:n] = np.array(rows, dtype=np.uint64).astype(np.uint32)
    inp = torch.from_numpy(arr.view(np.int32).reshape(-1).copy())
    out = torch.zeros(N * 4, dtype=torch.int32)
    _philox_rows[(1,)](inp, out, N=N)
    res = out.numpy().view(np.uint32).reshape(N, 4)[:n]
    print(json.dumps(res.astype(np.uint64).tolist()))


if __name__ == "__main__":
    main()
