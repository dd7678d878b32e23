"""Time one kernel of the library: python -m paper_1904_09538_gb300.runkernel
KERNEL key=value ... [--trials T] [--warmup W] [--flush]

Buffers are allocated per pm_kernel_buffers and filled with seeded uniform
values in [-1, 1) (bf16 buffers with random bit patterns of magnitude < 1).
Prints one JSON line: kernel, params, mean/median/min ms, algorithmic GB/s
and TFLOP/s where the counts define them."""
import json
import sys

import numpy as np
import torch

from . import kernel_buffers, run, counts


def main(argv):
    kernel, params, trials, warmup, flush = None, {}, 10, 3, False
    it = iter(argv)
    for a in it:
        if a == "--trials":
            trials = int(next(it))
        elif a == "--warmup":
            warmup = int(next(it))
        elif a == "--flush":
            flush = True
        elif "=" in a:
            k, v = a.split("=", 1)
            params[k] = float(v)
        else:
            kernel = a
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    bufs, nbytes = [], 0
    for b in kernel_buffers(kernel, **params):
        n = int(b["elems"])
        if b["dtype"] == np.uint16:
            x = (torch.randint(0, 1 << 14, (n,), device=dev, generator=gen, dtype=torch.int32) + 0x3800).to(torch.int16)
            nbytes += 2 * n
        elif b["dtype"] == np.float64:
            x = torch.rand(n, device=dev, generator=gen, dtype=torch.float64) * 2 - 1
            nbytes += 8 * n
        else:
            x = torch.rand(n, device=dev, generator=gen) * 2 - 1
            nbytes += 4 * n
        bufs.append(x)
    tm = run(kernel, bufs, warmup=warmup, trials=trials, flush_l2=flush, **params)
    flops = 0
    for r in counts(kernel, **params):
        if r["kind"] == "op":
            flops += r["count_wi"] * (2 if r["op"] == "madd" else 1)
    s = tm["mean_ms"] * 1e-3
    out = dict(kernel=kernel, params=params, mean_ms=tm["mean_ms"], median_ms=tm["median_ms"], min_ms=tm["min_ms"],
               buffer_GBps=nbytes / s / 1e9, TFLOPs=flops / s / 1e12)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1:])
