"""Measure this GPU's L2 and DRAM read bandwidth with the library's probe.

    python -m paper_2208_05247_b300.mem_probe [--sizes-mb 8 16 ...] [--out file.json]

For each buffer size the probe kernel (rt_probe_read) re-reads the buffer
with L2-cached 16-byte loads; the time per launch comes from CUDA events on
the current stream (best of 5 after warm-up). Below the L2 capacity the
rate is the L2 read bandwidth, above it the DRAM bandwidth; the size where
it falls is the effective L2 capacity for a streaming read. Prints one JSON
object: the sweep, the plateau below 64 MB (L2) and the rate at the largest
size (DRAM).
"""
from __future__ import annotations

import argparse
import json

from . import build, rt

SIZES_MB = (4, 8, 16, 32, 48, 64, 80, 96, 112, 128, 160, 192, 256, 512, 1024)


def sweep(sizes_mb=SIZES_MB, target_bytes=8 << 30, repeats=5):
    import torch
    big = max(sizes_mb) << 20
    buf = torch.ones(big // 4, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    out = []
    for mb in sizes_mb:
        nbytes = mb << 20
        reps = max(1, target_bytes // nbytes)
        rt.rt_probe_read(buf, nbytes, reps, sink, stream)          # warm-up (and fills L2)
        best = None
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rt.rt_probe_read(buf, nbytes, reps, sink, stream)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out.append({"mb": mb, "reps": reps, "ms": best, "gbs": nbytes * reps / (best * 1e-3) / 1e9})
    return out


def summary(rows):
    l2 = max(r["gbs"] for r in rows if r["mb"] <= 64)
    dram = rows[-1]["gbs"]
    knee = next((r["mb"] for r in rows if r["gbs"] < 0.5 * (l2 + dram)), None)
    return {"l2_read_gbs": l2, "dram_read_gbs": dram, "half_way_mb": knee}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--sizes-mb", type=int, nargs="+", default=SIZES_MB)
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    build.build()
    rows = sweep(tuple(a.sizes_mb))
    res = {"sweep": rows, **summary(rows)}
    print(json.dumps(res), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    return res


if __name__ == "__main__":
    main()
