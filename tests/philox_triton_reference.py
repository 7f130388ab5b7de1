"""Philox4x32-10 outputs from Triton's own implementation, run on the CPU by its
interpreter.  Used only as an independent reference for the oracle's Philox.
Prints one line per input: c0 c1 c2 c3 seed -> four output words (hex)."""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"
import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, n: tl.constexpr):
    o = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0_ptr + o), tl.load(c1_ptr + o), tl.load(c2_ptr + o),
                           tl.load(c3_ptr + o), 10)
    tl.store(out_ptr + 4 * o + 0, a)
    tl.store(out_ptr + 4 * o + 1, b)
    tl.store(out_ptr + 4 * o + 2, c)
    tl.store(out_ptr + 4 * o + 3, d)


def main():
    rows = [list(map(lambda s: int(s, 0), line.split())) for line in sys.stdin if line.strip()]
    by_seed = {}
    for r in rows:
        by_seed.setdefault(r[4], []).append(r)
    for seed, rs in by_seed.items():
        n = 1
        while n < len(rs):
            n *= 2
        cs = [torch.zeros(n, dtype=torch.uint32) for _ in range(4)]
        for i, r in enumerate(rs):
            for k in range(4):
                cs[k][i] = r[k]
        out = torch.zeros(4 * n, dtype=torch.uint32)
        _kernel[(1,)](out, *cs, seed, n)
        for i, r in enumerate(rs):
            words = [int(out[4 * i + k].item()) & 0xffffffff for k in range(4)]
            print(" ".join(hex(v) for v in r), "->", " ".join(hex(v) for v in words))


if __name__ == "__main__":
    main()
