"""FP64 numpy reference of the denoiser's layers (TEST INFRASTRUCTURE).

Only the tests use it, to check the BF16 tensor-core kernels of the denoiser.
Everything is written from the definitions, with no blocking or reordering:

  convolution   out[n,z,y,x,o] = b[o] + sum_{t,i} in[n, z+dz_t, y+dy_t, x+dx_t, i] W[t,i,o]
                (zero outside the volume; 3x3x3 taps ordered t = 9(dz+1) + 3(dy+1) + (dx+1),
                or one tap for 1x1x1)
  its gradients  d in, d W, d b from the chain rule of the same sum
  pooling       2x2x2 mean; upsampling: nearest neighbour (and their adjoints)
  loss          mean over voxels and used channels of w_c (pred - target)^2

Tensors are channels last: [N, D, H, W, C].
"""
from __future__ import annotations

import numpy as np


def taps(ksize: int):
    if ksize == 1:
        return [(0, 0, 0)]
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shifted(x, dz, dy, dx):
    """y[n,z,y,x,:] = x[n, z+dz, y+dy, x+dx, :] with zeros outside."""
    N, D, H, W, C = x.shape
    out = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), min(D, D - dz)), slice(max(0, -dy), min(H, H - dy)), slice(max(0, -dx), min(W, W - dx))
    zt, yt, xt = slice(max(0, dz), min(D, D + dz)), slice(max(0, dy), min(H, H + dy)), slice(max(0, dx), min(W, W + dx))
    out[:, zs, ys, xs, :] = x[:, zt, yt, xt, :]
    return out


def conv3d(x, W, b=None, ksize=3, relu=False):
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    out = np.zeros(x.shape[:4] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(taps(ksize)):
        out += _shifted(x, dz, dy, dx) @ W[t]
    if b is not None:
        out += np.asarray(b, np.float64)
    if relu:
        out = np.maximum(out, 0.0)
    return out


def conv3d_backward(x, W, gout, ksize=3):
    """Gradients of sum(gout * conv3d(x, W, b)) with respect to x, W and b."""
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    gout = np.asarray(gout, np.float64)
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t, (dz, dy, dx) in enumerate(taps(ksize)):
        xs = _shifted(x, dz, dy, dx)
        gW[t] = np.einsum("nzyxi,nzyxo->io", xs, gout)
        # adjoint of the shift: move gout back by (dz, dy, dx)
        gx += _shifted(gout @ W[t].T, -dz, -dy, -dx)
    gb = gout.sum(axis=(0, 1, 2, 3))
    return gx, gW, gb


def pool2(x):
    N, D, H, W, C = x.shape
    return np.asarray(x, np.float64).reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_backward(gout):
    return np.repeat(np.repeat(np.repeat(np.asarray(gout, np.float64), 2, 1), 2, 2), 2, 3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(np.asarray(x, np.float64), 2, 1), 2, 2), 2, 3)


def up2_backward(gout):
    N, D, H, W, C = gout.shape
    return np.asarray(gout, np.float64).reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def mse(pred, target, chw=None):
    """Loss and its gradient with respect to pred (channels of target only)."""
    pred = np.asarray(pred, np.float64)
    target = np.asarray(target, np.float64)
    C = target.shape[-1]
    w = np.ones(C) if chw is None else np.asarray(chw, np.float64)
    d = pred[..., :C] - target
    count = d.size
    loss = float((w * d * d).sum() / count)
    g = np.zeros_like(pred)
    g[..., :C] = 2.0 * w * d / count
    return loss, g


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((u >> 16) & 1)
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
