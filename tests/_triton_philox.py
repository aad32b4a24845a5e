"""Helper run in a subprocess: Philox4x32-10 words from Triton's own implementation
(``tl.philox``), executed by Triton's CPU interpreter. Reads JSON
{"ctr": [[c0,c1,c2,c3],...], "key": [k0,k1]} on stdin, writes JSON words on stdout.
Used only as an independent pin of the oracle's Philox."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kern(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c0p + offs)
    c1 = tl.load(c1p + offs)
    c2 = tl.load(c2p + offs)
    c3 = tl.load(c3p + offs)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(o0 + offs, r0)
    tl.store(o1 + offs, r1)
    tl.store(o2 + offs, r2)
    tl.store(o3 + offs, r3)


def main():
    req = json.load(sys.stdin)
    ctr = req["ctr"]
    n = len(ctr)
    m = 1
    while m < n:
        m *= 2
    cols = [torch.tensor([c[j] for c in ctr] + [0] * (m - n), dtype=torch.int64).to(torch.uint32) for j in range(4)]
    outs = [torch.zeros(m, dtype=torch.uint32) for _ in range(4)]
    seed = int(req["key"][0]) | (int(req["key"][1]) << 32)
    _kern[(1,)](seed, *cols, *outs, n=m)
    words = [[int(outs[j][i].to(torch.int64)) & 0xFFFFFFFF for j in range(4)] for i in range(n)]
    json.dump(words, sys.stdout)


if __name__ == "__main__":
    main()
