"""Time the denoiser's 3x3x3 convolution kernels on one layer shape.

    python -m paper_2208_05247_b300.conv_bench --shape 128 128 128 --cin 32 --cout 32 [--path tcgen05]
    python -m paper_2208_05247_b300.conv_bench --unet 128
    python -m paper_2208_05247_b300.conv_bench --layers 128
    python -m paper_2208_05247_b300.conv_bench --wgrad 128
    python -m paper_2208_05247_b300.conv_bench --unet-forward 128
    python -m paper_2208_05247_b300.conv_bench --pack 128

Prints one JSON line per kernel: CUDA-event time per launch (after warm-up, on
the current stream) and the dense FLOP rate 2 * 27 * Cin * Cout * voxels / t.
With --unet D it times the whole U-Net forward and backward at D^3 instead;
with --layers D every 3x3x3 layer shape of the U-Net's forward pass and input
gradients at D^3, with the mma.sync kernel, the per-tap tcgen05 kernel and the
default tcgen05 choice (halo-tiled where it fits); with --wgrad D the weight
gradient of every 3x3x3 forward layer at D^3 (mma.sync and tcgen05; the same
2 * 27 * Cin * Cout * voxels FLOPs); with --unet-forward D three untimed and
one timed forward pass of the U-Net (default kernels; for launch lists); with
--pack D the input packing and output unpacking of the denoiser at D^3.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import build, nn

PATHS = {"mma.sync": nn.NN_CONV_MMA_SYNC, "tcgen05": nn.NN_CONV_TCGEN05, "tcgen05-tap": nn.NN_CONV_TCGEN05_TAP,
         "tcgen05-halo": nn.NN_CONV_TCGEN05_HALO, "auto": nn.NN_CONV_AUTO}


def time_layer(shape, cin, cout, path, reps=10, warmup=3, relu=True):
    import torch
    vox = int(np.prod(shape))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(vox * cin, device="cuda", generator=g).to(torch.bfloat16)
    wt = (torch.randn(27 * cin * cout, device="cuda", generator=g) * 0.05).to(torch.bfloat16)
    out = torch.empty(vox * cout, dtype=torch.bfloat16, device="cuda")
    old = nn.nn_set_conv_path(PATHS[path])
    try:
        for _ in range(warmup):
            nn.nn_conv3d_fwd(x, wt, None, out, None, 1, *shape, cin, cout, 3, relu)
        ms = None
        for _ in range(3):                     # best of three timed blocks
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                nn.nn_conv3d_fwd(x, wt, None, out, None, 1, *shape, cin, cout, 3, relu)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / reps
            ms = t if ms is None else min(ms, t)
        nn.nn_status()
    finally:
        nn.nn_set_conv_path(old)
    return {"kernel": path, "shape": list(shape), "cin": cin, "cout": cout, "us": 1e3 * ms,
            "tflops": 2.0 * 27 * cin * cout * vox / (ms * 1e-3) / 1e12}


def time_wgrad(shape, cin, cout, path, reps=10, warmup=3):
    import torch
    vox = int(np.prod(shape))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(vox * cin, device="cuda", generator=g).to(torch.bfloat16)
    gy = torch.randn(vox * cout, device="cuda", generator=g).to(torch.bfloat16)
    gw = torch.zeros(27 * cin * cout, dtype=torch.float32, device="cuda")
    gb = torch.zeros(cout, dtype=torch.float32, device="cuda")
    old = nn.nn_set_conv_path(PATHS[path])
    try:
        for _ in range(warmup):
            nn.nn_conv3d_wgrad(x, gy, gw, gb, 1, *shape, cin, cout, 3)
        ms = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                nn.nn_conv3d_wgrad(x, gy, gw, gb, 1, *shape, cin, cout, 3)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / reps
            ms = t if ms is None else min(ms, t)
        nn.nn_status()
    finally:
        nn.nn_set_conv_path(old)
    return {"wgrad": path, "shape": list(shape), "cin": cin, "cout": cout, "us": 1e3 * ms,
            "tflops": 2.0 * 27 * cin * cout * vox / (ms * 1e-3) / 1e12}


def time_unet(d, path, reps=3):
    import torch
    from . import denoise
    net = denoise.UNet(seed=0)
    shape = (d, d, d)
    x = torch.randn(d ** 3 * denoise.CIN, device="cuda").to(torch.bfloat16)
    old = nn.nn_set_conv_path(PATHS[path])
    try:
        for _ in range(2):
            net.forward(x, shape)
            net.backward(x, shape)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd = bwd = 0.0
        for _ in range(reps):
            ev[0].record()
            net.forward(x, shape)
            ev[1].record()
            net.backward(x, shape)
            ev[2].record()
            torch.cuda.synchronize()
            fwd += ev[0].elapsed_time(ev[1])
            bwd += ev[1].elapsed_time(ev[2])
        nn.nn_status()
    finally:
        nn.nn_set_conv_path(old)
    return {"kernel": path, "unet": d, "forward_ms": fwd / reps, "backward_ms": bwd / reps,
            "forward_tflops": net.flops(shape) / (fwd / reps * 1e-3) / 1e12}


def unet_forward(d):
    """Three untimed forward passes and one timed one (CUDA events)."""
    import torch
    from . import denoise
    net = denoise.UNet(seed=0)
    shape = (d, d, d)
    x = torch.randn(d ** 3 * denoise.CIN, device="cuda").to(torch.bfloat16)
    for _ in range(3):
        net.forward(x, shape)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    net.forward(x, shape)
    b.record()
    torch.cuda.synchronize()
    nn.nn_status()
    return {"unet_forward": d, "ms": a.elapsed_time(b)}


def time_pack(d, reps=20):
    """CUDA-event time of nn_pack_inputs and nn_unpack at d^3 (best of 3 blocks)."""
    import torch
    from . import denoise
    n3, n2 = d ** 3, d ** 2
    g = torch.Generator(device="cuda").manual_seed(0)
    r = lambda n, dt=torch.float32: torch.rand(n, device="cuda", generator=g).to(dt)   # noqa: E731
    abs3d, sdir, sdif = r(n3, torch.float64), r(n2, torch.float64), r(n2, torch.float64)
    opt = [r(n3) for _ in range(5)]
    x = torch.empty(n3 * denoise.CIN, dtype=torch.bfloat16, device="cuda")
    pred = r(n3 * denoise.COUT)
    o3, o1, o2 = r(n3, torch.float64), r(n2, torch.float64), r(n2, torch.float64)
    out = {}
    for name, fn in (("pack_ms", lambda: nn.nn_pack_inputs(abs3d, sdir, sdif, *opt, x, d, d, d, 25.0, 866.0)),
                     ("unpack_ms", lambda: nn.nn_unpack(x, pred, denoise.COUT, o3, o1, o2, d, d, d, 25.0, 866.0))):
        for _ in range(3):
            fn()
        best = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / reps
            best = t if best is None else min(best, t)
        out[name] = best
    return {"pack": d, **out}


def unet_layers(d):
    """(shape, Cin, Cout) of the U-Net's 3x3x3 forward convolutions and input
    gradients at d^3 (an input gradient is a convolution with Cin and Cout swapped)."""
    from . import denoise
    c0, c1, c2, c3 = denoise.LEVELS
    fwd = [(0, denoise.CIN, c0), (0, c0, c0), (1, c0, c1), (1, c1, c1), (2, c1, c2), (2, c2, c2), (3, c2, c3),
           (3, c3, c3), (2, c3 + c2, c2), (1, c2 + c1, c1), (0, c1 + c0, c0)]
    out, seen = [], set()
    for lvl, a, b in fwd + [(lvl, b, a) for lvl, a, b in fwd]:
        key = (lvl, a, b)
        if key not in seen:
            seen.add(key)
            out.append(((d >> lvl,) * 3, a, b))
    return out


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--shape", type=int, nargs=3, default=(128, 128, 128), help="D H W")
    p.add_argument("--cin", type=int, default=32)
    p.add_argument("--cout", type=int, default=32)
    p.add_argument("--path", choices=sorted(PATHS), default=None, help="one kernel (default: mma.sync and tcgen05)")
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--bwd", action="store_true", help="time the weight gradient of --shape instead")
    p.add_argument("--unet", type=int, default=0, help="time the whole U-Net at this edge length instead")
    p.add_argument("--layers", type=int, default=0, help="time every U-Net layer shape at this edge length")
    p.add_argument("--wgrad", type=int, default=0, help="time every U-Net weight gradient at this edge length")
    p.add_argument("--unet-forward", type=int, default=0, help="3 untimed + 1 timed U-Net forward at this edge length")
    p.add_argument("--pack", type=int, default=0, help="time the denoiser's input packing and unpacking at this edge")
    a = p.parse_args(argv)
    build.build()
    if a.pack:
        print(json.dumps(time_pack(a.pack)), flush=True)
        return
    if a.unet_forward:
        print(json.dumps(unet_forward(a.unet_forward)), flush=True)
        return
    if a.wgrad:
        for shape, cin, cout in unet_layers(a.wgrad)[:11]:
            for path in ("mma.sync", "tcgen05"):
                print(json.dumps(time_wgrad(shape, cin, cout, path, reps=a.reps)), flush=True)
        return
    if a.layers:
        for shape, cin, cout in unet_layers(a.layers):
            for path in ("mma.sync", "tcgen05-tap", "tcgen05"):
                print(json.dumps(time_layer(shape, cin, cout, path, reps=a.reps)), flush=True)
        return
    paths = [a.path] if a.path else (["mma.sync", "tcgen05"] if not a.unet else ["mma.sync", "tcgen05-tap", "auto"])
    for path in paths:
        if a.unet:
            r = time_unet(a.unet, path)
        elif a.bwd:
            r = time_wgrad(tuple(a.shape), a.cin, a.cout, path, reps=a.reps)
        else:
            r = time_layer(tuple(a.shape), a.cin, a.cout, path, reps=a.reps)
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
