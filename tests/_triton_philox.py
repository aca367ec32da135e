"""Philox-4x32-10 from Triton's ``tl.philox`` run by Triton's CPU interpreter.

Used only as an independent library reference for the oracle's Philox.
Run as a subprocess: reads a .npy of [n, 6] uint32 rows (key0, key1, c0..c3)
and writes a .npy of [n, 4] uint32 outputs."""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    mask = offs < n
    c0 = tl.load(c0_ptr + offs, mask=mask).to(tl.uint32, bitcast=True)
    c1 = tl.load(c1_ptr + offs, mask=mask).to(tl.uint32, bitcast=True)
    c2 = tl.load(c2_ptr + offs, mask=mask).to(tl.uint32, bitcast=True)
    c3 = tl.load(c3_ptr + offs, mask=mask).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * offs + 0, a.to(tl.int32, bitcast=True), mask=mask)
    tl.store(out_ptr + 4 * offs + 1, b.to(tl.int32, bitcast=True), mask=mask)
    tl.store(out_ptr + 4 * offs + 2, c.to(tl.int32, bitcast=True), mask=mask)
    tl.store(out_ptr + 4 * offs + 3, d.to(tl.int32, bitcast=True), mask=mask)


def main(src, dst):
    rows = np.load(src).astype(np.uint32)
    out = np.zeros((len(rows), 4), np.uint32)
    for i, r in enumerate(rows):
        seed = int(r[0]) | (int(r[1]) << 32)
        cs = [torch.tensor([int(v)], dtype=torch.int64).to(torch.int32) if v < 2**31
              else torch.tensor([int(v) - 2**32], dtype=torch.int32) for v in r[2:6]]
        o = torch.zeros(4, dtype=torch.int32)
        _kernel[(1,)](o, cs[0], cs[1], cs[2], cs[3], seed, 1, BLOCK=1)
        out[i] = o.numpy().view(np.uint32)
    np.save(dst, out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
