"""Philox4x32-10 words from Triton's own implementation, run on the CPU through
Triton's interpreter.  Used only as an independent reference for the oracle's
generator; prints a JSON list of [counter, key, words] triples."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402,F401
import triton.language as tl  # noqa: E402
from triton.language.random import philox  # noqa: E402


@triton.jit
def _kernel(out_ptr, c_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)


def main():
    seeds = [int(s) for s in sys.argv[1:]] or [0, 1, 0x1234567890ABCDEF]
    rng = np.random.default_rng(2024)
    out = []
    for seed in seeds:
        ctr = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = [1, 0, 0, 0]
        ctr[2] = [0xFFFFFFFF] * 4
        res = torch.zeros(16 * 4, dtype=torch.int32)
        _kernel[(1,)](res, torch.from_numpy(ctr.view(np.int32).copy()), seed, 16)
        words = res.view(16, 4).numpy().view(np.uint32)
        for c, w in zip(ctr, words):
            out.append([[int(x) for x in c], [seed & 0xFFFFFFFF, seed >> 32], [int(x) for x in w]])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
