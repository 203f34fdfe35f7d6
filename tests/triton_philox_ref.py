"""Independent Philox4x32-10 words from Triton's CPU interpreter.

Run as a subprocess with TRITON_INTERPRET=1 (set below, before the import).
Reads JSON {"cases": [[seed, c0, c1, c2, c3], ...]} on stdin and prints the
four 32-bit output words of each case as JSON. Triton's ``tl.philox`` keys
the generator with (seed_lo, seed_hi) and runs 10 rounds by default; it is
used here only as a library implementation of the published generator to pin
the oracle against something other than itself.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + i * 4 + 0)
    c1 = tl.load(c_ptr + i * 4 + 1)
    c2 = tl.load(c_ptr + i * 4 + 2)
    c3 = tl.load(c_ptr + i * 4 + 3)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, r0.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 1, r1.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 2, r2.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 3, r3.to(tl.int32, bitcast=True))


def main():
    cases = json.load(sys.stdin)["cases"]
    out = []
    for seed, *ctr in cases:
        c = torch.tensor([[x - (1 << 32) if x >= (1 << 31) else x for x in ctr]], dtype=torch.int32)
        c = torch.cat([c, torch.zeros((1, 4), dtype=torch.int32)], 0).reshape(-1)
        o = torch.zeros(8, dtype=torch.int32)
        _philox_kernel[(1,)](c, o, seed, 2)
        out.append([int(v) & 0xFFFFFFFF for v in o[:4].tolist()])
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
