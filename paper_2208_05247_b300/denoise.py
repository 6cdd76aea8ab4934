"""Learned denoiser for low-photon ray-traced fields (3D U-Net, BF16 tensor cores).

The paper's tracer error falls as N^-1/2 with the photon count while the cost
grows as N (Sec. 3.2). This module trains a network that maps a field traced
with few photons per column (plus the optics) to the field a high photon count
gives, and measures whether tracing few photons and denoising reaches a given
RMS error in less wall time than tracing more photons.

Network: 4-level 3D U-Net, 32 base channels (32, 64, 128, 256), two 3x3x3
convolutions + ReLU per level, 2x2x2 average pooling down, nearest 2x
upsampling + concatenation up, a 1x1x1 head to 16 channels of which 3 are used
(corrections to the noisy absorption and surface direct/diffuse channels).
BF16 weights and activations, FP32 accumulation and FP32 master weights; Adam.
Every forward, backward and optimizer operation runs in the library's kernels
(include/nn.h); torch only holds the device buffers.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import nn, rt, scenes

CIN = 16      # packed input channels (6 used; 8 with the direct-beam features)
COUT = 16     # head channels (3 used)
NUSE = 3
LEVELS = (32, 64, 128, 256)


def _torch():
    import torch
    return torch


class Conv:
    """One convolution layer: FP32 master weights, BF16 copies, Adam state."""

    def __init__(self, cin, cout, ksize, relu, rng, dev):
        torch = _torch()
        self.cin, self.cout, self.ksize, self.relu = cin, cout, ksize, relu
        taps = 27 if ksize == 3 else 1
        std = math.sqrt(2.0 / (taps * cin)) if relu else math.sqrt(1.0 / (taps * cin)) * 0.1
        w = rng.normal(0.0, std, size=(taps, cin, cout)).astype(np.float32)
        self.W = torch.from_numpy(w).to(dev)
        self.b = torch.zeros(cout, dtype=torch.float32, device=dev)
        self.gW = torch.zeros_like(self.W)
        self.gb = torch.zeros_like(self.b)
        self.mW, self.vW = torch.zeros_like(self.W), torch.zeros_like(self.W)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.wt = torch.empty(self.W.numel(), dtype=torch.bfloat16, device=dev)
        self.wd = torch.empty_like(self.wt)
        self.We, self.be = self.W.clone(), self.b.clone()     # moving averages
        self.refresh()

    def refresh(self, stream=None):
        nn.nn_weights_bf16(self.W, self.wt, self.wd, self.ksize, self.cin, self.cout, stream)

    def forward(self, x, shape, out_bf16=None, out_f32=None, stream=None):
        nn.nn_conv3d_fwd(x, self.wt, self.b, out_bf16, out_f32, 1, *shape, self.cin, self.cout, self.ksize,
                         self.relu, stream)

    def backward(self, x, y, gy, gx, shape, stream=None):
        """gy: gradient at this layer's output (modified in place by the ReLU mask)."""
        if self.relu:
            nn.nn_relu_bwd(y, gy, stream)
        nn.nn_conv3d_wgrad(x, gy, self.gW, self.gb, 1, *shape, self.cin, self.cout, self.ksize, stream)
        if gx is not None:
            nn.nn_conv3d_fwd(gy, self.wd, None, gx, None, 1, *shape, self.cout, self.cin, self.ksize, False, stream)

    def step(self, lr, t, weight_decay=0.0, stream=None):
        nn.nn_adam(self.W, self.mW, self.vW, self.gW, lr, t, weight_decay=weight_decay, stream=stream)
        nn.nn_adam(self.b, self.mb, self.vb, self.gb, lr, t, stream=stream)
        self.refresh(stream)

    def ema(self, decay, stream=None):
        nn.nn_ema(self.We, self.W, decay, stream)
        nn.nn_ema(self.be, self.b, decay, stream)

    def apply_ema(self):
        self.W.copy_(self.We)
        self.b.copy_(self.be)
        self.refresh()

    def rollback(self):
        """Back to the averaged weights with fresh Adam moments."""
        self.apply_ema()
        for t in (self.mW, self.vW, self.mb, self.vb):
            t.zero_()

    def state(self):
        return {"W": self.W.cpu().numpy(), "b": self.b.cpu().numpy()}

    def load(self, st):
        torch = _torch()
        self.W.copy_(torch.from_numpy(st["W"]))
        self.b.copy_(torch.from_numpy(st["b"]))
        self.refresh()


class UNet:
    """4-level 3D U-Net over [D][H][W][16] inputs; D, H, W divisible by 8."""

    def __init__(self, seed=0, device="cuda"):
        rng = np.random.default_rng(seed)
        c0, c1, c2, c3 = LEVELS
        mk = lambda a, b, k=3, r=True: Conv(a, b, k, r, rng, device)   # noqa: E731
        self.enc = [(mk(CIN, c0), mk(c0, c0)), (mk(c0, c1), mk(c1, c1)), (mk(c1, c2), mk(c2, c2)),
                    (mk(c2, c3), mk(c3, c3))]
        self.dec = [(mk(c3 + c2, c2), mk(c2, c2)), (mk(c2 + c1, c1), mk(c1, c1)), (mk(c1 + c0, c0), mk(c0, c0))]
        self.head = mk(c0, COUT, 1, False)
        self.device = device
        self.t = 0
        self._buf = {}

    def layers(self):
        return [c for pair in self.enc + self.dec for c in pair] + [self.head]

    def n_params(self):
        return sum(c.W.numel() + c.b.numel() for c in self.layers())

    def flops(self, shape):
        """Multiply-adds x 2 of one forward pass."""
        D, H, W = shape
        total = 0
        sizes = [D * H * W // 8 ** lvl for lvl in range(4)]
        for lvl, (a, b) in enumerate(self.enc):
            total += 2 * sizes[lvl] * (27 * a.cin * a.cout + 27 * b.cin * b.cout)
        for k, (a, b) in enumerate(self.dec):
            total += 2 * sizes[2 - k] * (27 * a.cin * a.cout + 27 * b.cin * b.cout)
        return total + 2 * sizes[0] * self.head.cin * self.head.cout

    # ---- buffers ---------------------------------------------------------------
    def _buffers(self, shape):
        if shape in self._buf:
            return self._buf[shape]
        torch = _torch()
        D, H, W = shape
        V = [D * H * W // 8 ** lvl for lvl in range(4)]
        c0, c1, c2, c3 = LEVELS
        bf = lambda n: torch.empty(n, dtype=torch.bfloat16, device=self.device)  # noqa: E731
        B = {"V": V}
        for name, lvl, c in (("a0", 0, c0), ("e0", 0, c0), ("p0", 1, c0), ("a1", 1, c1), ("e1", 1, c1),
                             ("p1", 2, c1), ("a2", 2, c2), ("e2", 2, c2), ("p2", 3, c2), ("a3", 3, c3),
                             ("b3", 3, c3), ("cat2", 2, c3 + c2), ("d2a", 2, c2), ("d2", 2, c2),
                             ("cat1", 1, c2 + c1), ("d1a", 1, c1), ("d1", 1, c1), ("cat0", 0, c1 + c0),
                             ("d0a", 0, c0), ("d0", 0, c0)):
            B[name] = bf(V[lvl] * c)
            B["g_" + name] = bf(V[lvl] * c)
        B["tmp0"], B["tmp1"], B["tmp2"] = bf(V[0] * c0), bf(V[1] * c1), bf(V[2] * c2)
        B["out"] = torch.empty(V[0] * COUT, dtype=torch.float32, device=self.device)
        B["g_out"] = bf(V[0] * COUT)
        B["loss"] = torch.zeros(1, dtype=torch.float64, device=self.device)
        self._buf[shape] = B
        return B

    # ---- passes ----------------------------------------------------------------
    def forward(self, x, shape, stream=None):
        """x: BF16 [D*H*W*16]; returns the FP32 head output [D*H*W*16] (a buffer)."""
        B = self._buffers(shape)
        D, H, W = shape
        s = [(D >> l, H >> l, W >> l) for l in range(4)]
        V = B["V"]
        c0, c1, c2, c3 = LEVELS
        (e0a, e0b), (e1a, e1b), (e2a, e2b), (ba, bb) = self.enc
        e0a.forward(x, s[0], B["a0"], stream=stream); e0b.forward(B["a0"], s[0], B["e0"], stream=stream)
        nn.nn_pool2_fwd(B["e0"], B["p0"], 1, *s[0], c0, stream)
        e1a.forward(B["p0"], s[1], B["a1"], stream=stream); e1b.forward(B["a1"], s[1], B["e1"], stream=stream)
        nn.nn_pool2_fwd(B["e1"], B["p1"], 1, *s[1], c1, stream)
        e2a.forward(B["p1"], s[2], B["a2"], stream=stream); e2b.forward(B["a2"], s[2], B["e2"], stream=stream)
        nn.nn_pool2_fwd(B["e2"], B["p2"], 1, *s[2], c2, stream)
        ba.forward(B["p2"], s[3], B["a3"], stream=stream); bb.forward(B["a3"], s[3], B["b3"], stream=stream)
        (d2a, d2b), (d1a, d1b), (d0a, d0b) = self.dec
        nn.nn_up2_fwd(B["b3"], B["cat2"], 1, *s[3], c3, c3 + c2, 0, stream)
        nn.nn_copy_channels(B["e2"], c2, 0, B["cat2"], c3 + c2, c3, V[2], c2, False, stream)
        d2a.forward(B["cat2"], s[2], B["d2a"], stream=stream); d2b.forward(B["d2a"], s[2], B["d2"], stream=stream)
        nn.nn_up2_fwd(B["d2"], B["cat1"], 1, *s[2], c2, c2 + c1, 0, stream)
        nn.nn_copy_channels(B["e1"], c1, 0, B["cat1"], c2 + c1, c2, V[1], c1, False, stream)
        d1a.forward(B["cat1"], s[1], B["d1a"], stream=stream); d1b.forward(B["d1a"], s[1], B["d1"], stream=stream)
        nn.nn_up2_fwd(B["d1"], B["cat0"], 1, *s[1], c1, c1 + c0, 0, stream)
        nn.nn_copy_channels(B["e0"], c0, 0, B["cat0"], c1 + c0, c1, V[0], c0, False, stream)
        d0a.forward(B["cat0"], s[0], B["d0a"], stream=stream); d0b.forward(B["d0a"], s[0], B["d0"], stream=stream)
        self.head.forward(B["d0"], s[0], out_f32=B["out"], stream=stream)
        return B["out"]

    def backward(self, x, shape, stream=None):
        """Backward from B['g_out'] (written by the loss); accumulates layer gradients."""
        B = self._buffers(shape)
        D, H, W = shape
        s = [(D >> l, H >> l, W >> l) for l in range(4)]
        V = B["V"]
        c0, c1, c2, c3 = LEVELS
        for c in self.layers():
            c.gW.zero_()
            c.gb.zero_()
        (e0a, e0b), (e1a, e1b), (e2a, e2b), (ba, bb) = self.enc
        (d2a, d2b), (d1a, d1b), (d0a, d0b) = self.dec
        self.head.backward(B["d0"], None, B["g_out"], B["g_d0"], s[0], stream)
        d0b.backward(B["d0a"], B["d0"], B["g_d0"], B["g_d0a"], s[0], stream)
        d0a.backward(B["cat0"], B["d0a"], B["g_d0a"], B["g_cat0"], s[0], stream)
        nn.nn_up2_bwd(B["g_cat0"], B["g_d1"], 1, *s[1], c1, c1 + c0, 0, stream)
        nn.nn_copy_channels(B["g_cat0"], c1 + c0, c1, B["g_e0"], c0, 0, V[0], c0, False, stream)
        d1b.backward(B["d1a"], B["d1"], B["g_d1"], B["g_d1a"], s[1], stream)
        d1a.backward(B["cat1"], B["d1a"], B["g_d1a"], B["g_cat1"], s[1], stream)
        nn.nn_up2_bwd(B["g_cat1"], B["g_d2"], 1, *s[2], c2, c2 + c1, 0, stream)
        nn.nn_copy_channels(B["g_cat1"], c2 + c1, c2, B["g_e1"], c1, 0, V[1], c1, False, stream)
        d2b.backward(B["d2a"], B["d2"], B["g_d2"], B["g_d2a"], s[2], stream)
        d2a.backward(B["cat2"], B["d2a"], B["g_d2a"], B["g_cat2"], s[2], stream)
        nn.nn_up2_bwd(B["g_cat2"], B["g_b3"], 1, *s[3], c3, c3 + c2, 0, stream)
        nn.nn_copy_channels(B["g_cat2"], c3 + c2, c3, B["g_e2"], c2, 0, V[2], c2, False, stream)
        bb.backward(B["a3"], B["b3"], B["g_b3"], B["g_a3"], s[3], stream)
        ba.backward(B["p2"], B["a3"], B["g_a3"], B["g_p2"], s[3], stream)
        nn.nn_pool2_bwd(B["g_p2"], B["tmp2"], 1, *s[2], c2, stream)
        nn.nn_copy_channels(B["tmp2"], c2, 0, B["g_e2"], c2, 0, V[2], c2, True, stream)
        e2b.backward(B["a2"], B["e2"], B["g_e2"], B["g_a2"], s[2], stream)
        e2a.backward(B["p1"], B["a2"], B["g_a2"], B["g_p1"], s[2], stream)
        nn.nn_pool2_bwd(B["g_p1"], B["tmp1"], 1, *s[1], c1, stream)
        nn.nn_copy_channels(B["tmp1"], c1, 0, B["g_e1"], c1, 0, V[1], c1, True, stream)
        e1b.backward(B["a1"], B["e1"], B["g_e1"], B["g_a1"], s[1], stream)
        e1a.backward(B["p0"], B["a1"], B["g_a1"], B["g_p0"], s[1], stream)
        nn.nn_pool2_bwd(B["g_p0"], B["tmp0"], 1, *s[0], c0, stream)
        nn.nn_copy_channels(B["tmp0"], c0, 0, B["g_e0"], c0, 0, V[0], c0, True, stream)
        e0b.backward(B["a0"], B["e0"], B["g_e0"], B["g_a0"], s[0], stream)
        e0a.backward(x, B["a0"], B["g_a0"], None, s[0], stream)

    def loss_and_grad(self, target, shape, chw, stream=None):
        B = self._buffers(shape)
        B["loss"].zero_()
        nn.nn_mse(B["out"], COUT, target, NUSE, chw, B["g_out"], B["V"][0], B["loss"], stream)
        return B["loss"]

    def step(self, lr, weight_decay=0.0, stream=None):
        self.t += 1
        for c in self.layers():
            c.step(lr, self.t, weight_decay, stream)

    def ema(self, decay, stream=None):
        for c in self.layers():
            c.ema(decay, stream)

    def apply_ema(self):
        """Replace the weights by their moving averages."""
        for c in self.layers():
            c.apply_ema()

    def rollback(self):
        """Back to the averaged weights; Adam restarts (zero moments, step 0)."""
        self.t = 0
        for c in self.layers():
            c.rollback()

    def state(self):
        return [c.state() for c in self.layers()]

    def load(self, st):
        for c, s in zip(self.layers(), st):
            c.load(s)


# ---- pairs from the tracer -------------------------------------------------------------

@dataclass
class Sample:
    x: object          # BF16 [V*16] packed low-photon input
    target: object     # FP32 [V*3] correction to the input channels (None for evaluation inputs)
    shape: tuple
    flux: float        # toa_flux * cos(sza)
    dz: float


def _gen_scene(args):
    seed, nx, ny, nz = args
    return scenes.cumulus_scene(seed=seed, nx=nx, ny=ny, nz=nz)


def make_scenes(seeds, nx, ny, nz, workers=8):
    """Seeded cumulus scenes, generated in a spawned process pool."""
    import multiprocessing as mp
    args = [(s, nx, ny, nz) for s in seeds]
    if workers <= 1 or len(args) < 4:
        return [_gen_scene(a) for a in args]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen_scene, args, chunksize=max(1, len(args) // (4 * workers)))


class FieldTracer:
    """Traces scenes of one shape into device FP64 fields (handle reused).

    spectral=False traces one quadrature point (TOA flux 1000 W m^-2).
    spectral=True traces the broadband field the paper's heating rates and GHI
    are: all quadrature points of `scenes.gpoint_table()` (gas extinction scale
    and TOA flux per point, fluxes summing to 1000 W m^-2) in one batched launch,
    `ppc` photons per column per quadrature point on average, split in
    proportion to each point's energy (Sec. 2.3 traces every point
    independently; N_sample counts rays per column per point, Sec. 2.4).
    """

    def __init__(self, shape, dx=50.0, dy=50.0, dz=25.0, stream=None, spectral=False, direct_features=False):
        torch = _torch()
        nz, ny, nx = shape
        self.t = rt.Tracer(nx, ny, nz, dx, dy, dz, stream=stream)
        self.spectral = spectral
        if spectral:
            self.t.set_options(batch_optics=1)
            self.gas_scale, self.gflux = scenes.gpoint_table()
        self.shape = shape
        self.dz = dz
        dev = "cuda"
        self.ncell, self.ncol = nx * ny * nz, nx * ny
        self.optics = [torch.empty(self.ncell, dtype=torch.float32, device=dev) for _ in range(5)]
        self.alb = torch.empty(self.ncol, dtype=torch.float32, device=dev)
        # optional input channels 6 and 7: deterministic direct-beam transmittance
        # of each voxel (column centre) and the pixel-mean one at the surface.
        self.direct_features = direct_features
        self.t3d = torch.empty(self.ncell, dtype=torch.float32, device=dev)
        self.t2d = torch.empty(self.ncol, dtype=torch.float32, device=dev)
        self.t2s = torch.empty(self.ncol, dtype=torch.float32, device=dev)
        self.dx, self.dy = dx, dy

    def load(self, scene):
        torch = _torch()
        for dst, a in zip(self.optics, scene.fields()):
            dst.copy_(torch.from_numpy(np.ascontiguousarray(a).ravel()))
        self.alb.copy_(torch.from_numpy(scene.albedo.ravel()))
        self.t.set_optics(*self.optics)
        self.t.set_surface(self.alb)
        self.t.build_accel(2, 2, 2)

    def trace(self, sza, ppc, seed, out=None):
        """Trace ppc photons per column; returns device (abs3d, sfc_dir, sfc_dif) FP64."""
        torch = _torch()
        if out is None:
            out = (torch.empty(self.ncell, dtype=torch.float64, device="cuda"),
                   torch.empty(self.ncol, dtype=torch.float64, device="cuda"),
                   torch.empty(self.ncol, dtype=torch.float64, device="cuda"))
        self.t.reset()
        if self.spectral:
            jobs = [dict(scene=self.t, sza_deg=sza, toa_flux=float(f), gas_scale=float(g))
                    for g, f in zip(self.gas_scale, self.gflux)]
            rt.rt_trace_batch(jobs, total_photons=ppc * len(jobs) * self.ncol, seed=seed)
        else:
            self.t.trace(sza, 0.0, 1000.0, ppc * self.ncol, seed)
        rt.rt_fields(self.t.h, self.ncell, self.ncol, out[0], out[1], out[2], None)
        return out

    def pack(self, lo, sza, hi=None):
        torch = _torch()
        nz, ny, nx = self.shape
        F = 1000.0 * math.cos(math.radians(sza))
        x = torch.empty(self.ncell * CIN, dtype=torch.bfloat16, device="cuda")
        if self.direct_features:
            # deterministic direct-beam transmittance of the optics (input channels 6, 7)
            nn.nn_direct_transmittance(self.optics[0], self.optics[2], nz, ny, nx, self.dx, self.dy, self.dz, sza,
                                       0.0, self.t3d, self.t2d)
            nn.nn_direct_surface(self.optics[0], self.optics[2], nz, ny, nx, self.dx, self.dy, self.dz, sza, 0.0, 8,
                                 self.t2d)
        nn.nn_pack_inputs(lo[0], lo[1], lo[2], *self.optics, x, nz, ny, nx, self.dz, F,
                          t3d=self.t3d if self.direct_features else None,
                          t2d=self.t2d if self.direct_features else None)
        tgt = None
        if hi is not None:
            tgt = torch.empty(self.ncell * NUSE, dtype=torch.float32, device="cuda")
            nn.nn_pack_targets(hi[0], hi[1], hi[2], lo[0], lo[1], lo[2], tgt, nz, ny, nx, self.dz, F)
        return Sample(x, tgt, self.shape, F, self.dz)

    def direct_surface(self, sza, nsub=8, stream=None):
        """Expected surface direct irradiance [W m^-2], device FP64 [ny*nx]:
        toa_flux cos(sza) times the pixel-mean Beer-Lambert transmittance over
        nsub x nsub surface points per column (one quadrature point only).
        Runs on `stream` (a torch stream) if given, else on the current one."""
        torch = _torch()
        if self.spectral:
            raise ValueError("direct_surface covers the single quadrature point")
        nz, ny, nx = self.shape
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            nn.nn_direct_surface(self.optics[0], self.optics[2], nz, ny, nx, self.dx, self.dy, self.dz, sza, 0.0,
                                 nsub, self.t2s, torch.cuda.current_stream())
            return self.t2s.double() * (1000.0 * math.cos(math.radians(sza)))

    def close(self):
        self.t.close()


SZAS = (0.0, 30.0, 60.0)


def make_pairs(seeds, shape, lo_ppc=4, hi_ppc=1024, workers=8, spectral=False, direct_features=False):
    """Training pairs (low-photon input, correction target) traced on the GPU."""
    nz, ny, nx = shape
    scs = make_scenes(seeds, nx, ny, nz, workers)
    ft = FieldTracer(shape, spectral=spectral, direct_features=direct_features)
    out = []
    for seed, sc in zip(seeds, scs):
        sza = SZAS[seed % 3]
        ft.load(sc)
        lo = ft.trace(sza, lo_ppc, 2 * seed + 1)
        hi = ft.trace(sza, hi_ppc, 2 * seed + 2)
        out.append(ft.pack(lo, sza, hi))
    ft.close()
    return out


def channel_weights(samples, device="cuda", direct=True):
    """1 / variance of each target channel over the samples (balances the loss).
    direct=False drops the surface-direct channel from the loss: the denoised
    product then takes the exact direct beam (FieldTracer.direct_surface), and
    the network's capacity goes to absorption and diffuse irradiance."""
    torch = _torch()
    v = np.zeros(NUSE)
    for s in samples:
        t = s.target.view(-1, NUSE).double()
        v += (t * t).mean(0).cpu().numpy()
    v /= len(samples)
    w = 1.0 / np.maximum(v, 1e-12)
    if not direct:
        w[1] = 0.0
    return torch.tensor(w.astype(np.float32), device=device)


def train(net, samples, epochs=4, lr=1e-3, lr_final=1e-4, chw=None, log=None, seed=0, ema=True, warmup=0.05):
    """Adam over the samples (one scene per step), cosine learning-rate decay;
    the rate first rises linearly over the fraction `warmup` of the steps
    (0.05: two runs of the 512-scene configuration reached heating-rate errors
    of 0.069-0.071 K/day against 0.081-0.083 without it).

    With `ema` the returned network holds the moving average of its weights
    over roughly the last tenth of the steps (decay 1 - 10 / steps, capped
    at (1 + n) / (10 + n) after n updates so that the average follows the
    weights early on).

    Guards keep long runs from collapsing (a few runs diverged at full
    learning rate while repeats of the same run did not): a step whose loss
    is non-finite or above 8x the running mean loss is skipped; 32 skipped
    steps in a row (the weights themselves have diverged, so every loss is
    out of range) or a running mean above 4x its lowest value roll the
    weights back to their moving average with a fresh Adam state, and the
    learning-rate ramp starts again (a fresh Adam state takes full-size steps
    at once, and at full rate one run diverged again after every rollback).
    `net.train_log` records skips and rollbacks.
    """
    torch = _torch()
    rng = np.random.default_rng(seed)
    if chw is None:
        chw = channel_weights(samples)
    steps = epochs * len(samples)
    losses = []
    k = 0
    t0 = time.time()
    run, best, skipped, rollbacks, streak = None, None, 0, 0, 0
    ramp_from = 0                  # the learning-rate ramp restarts at every rollback
    n_avg = 0                      # updates of the moving average so far
    for ep in range(epochs):
        for idx in rng.permutation(len(samples)):
            s = samples[idx]
            net.forward(s.x, s.shape)
            loss = net.loss_and_grad(s.target, s.shape, chw)
            lv = float(loss.item())
            k += 1
            if not math.isfinite(lv) or (run is not None and k > 64 and lv > 8.0 * run):
                skipped += 1
                streak += 1
                if ema and streak >= 32:
                    net.rollback()
                    rollbacks += 1
                    streak = 0
                    ramp_from = k
                    # the averaged weights may sit above the old running mean
                    # and its lowest value: restart both, or every later step
                    # would be skipped or rolled back again
                    run = best = None
                continue
            streak = 0
            run = lv if run is None else 0.98 * run + 0.02 * lv
            if k > 256:
                best = run if best is None else min(best, run)
                if ema and run > 4.0 * best:
                    net.rollback()
                    rollbacks += 1
                    run = best = None
                    ramp_from = k
                    continue
            net.backward(s.x, s.shape)
            rate = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * (k - 1) / max(1, steps - 1)))
            if warmup > 0.0:
                rate *= min(1.0, (k - ramp_from) / max(1.0, warmup * steps))
            net.step(rate)
            if ema:
                # the average spans ~the last tenth of the steps at the end, and
                # only the updates so far early on (a rollback in the first
                # steps then returns to recent weights, not the initial ones)
                n_avg += 1
                net.ema(min(1.0 - 10.0 / max(steps, 20), (1.0 + n_avg) / (10.0 + n_avg)))
            if k % 16 == 0 or k == steps:
                losses.append((k, lv))
                if log:
                    log(f"step {k}/{steps} loss {lv:.4f} ({time.time() - t0:.0f}s)")
    if ema:
        net.apply_ema()
    net.train_log = {"skipped_steps": skipped, "rollbacks": rollbacks}
    torch.cuda.synchronize()
    if not losses:
        losses.append((k, run if run is not None else float("nan")))
    return losses


def denoise(net, sample):
    """Denoised fields (device FP64 abs3d, sfc_dir, sfc_dif) of a packed sample."""
    torch = _torch()
    nz, ny, nx = sample.shape
    out = net.forward(sample.x, sample.shape)
    abs3d = torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
    sd = torch.empty(ny * nx, dtype=torch.float64, device="cuda")
    sf = torch.empty(ny * nx, dtype=torch.float64, device="cuda")
    nn.nn_unpack(sample.x, out, COUT, abs3d, sd, sf, nz, ny, nx, sample.dz, sample.flux)
    return abs3d, sd, sf


# ---- evaluation: wall time to a target RMS error ----------------------------------------

def heating_factor(nz, dz):
    """K/day per W m^-3 per layer: 86400 / (rho(z) c_p), rho = 1.225 exp(-z/8000), c_p = 1004."""
    zc = (np.arange(nz) + 0.5) * dz
    return 86400.0 / (1.225 * np.exp(-zc / 8000.0) * 1004.0)


def plain_time_at(plain_ppc, ms, n):
    """Plain-tracer time at n photons/column from the measured runs, with no
    model: linear between the two runs around n; beyond the largest run,
    extended at the rate of the last two (the bulk rate of long launches);
    below the smallest, that run's time (a launch lasts at least as long as
    its longest history, whatever the photon count)."""
    runs = sorted(zip(plain_ppc, ms))
    if math.isinf(n):
        return math.inf
    if n <= runs[0][0]:
        return runs[0][1]
    for (p0, m0), (p1, m1) in zip(runs, runs[1:]):
        if n <= p1:
            return m0 + (m1 - m0) * (n - p0) / (p1 - p0)
    (p0, m0), (p1, m1) = runs[-2], runs[-1]
    return m1 + (m1 - m0) / (p1 - p0) * (n - p1)


def plain_time_fit(plain_ppc, ms):
    """Least-squares line time = t0 + t1 * ppc through the plain runs' times."""
    t1, t0 = np.polyfit(np.asarray(plain_ppc, dtype=np.float64), np.asarray(ms, dtype=np.float64), 1)
    return float(t0), float(t1)


def speedup_bracket(plain_ppc, rmse, ms, target, t_denoised, extra_ms=0.0):
    """Speed-up bounds that need no error or time model. The plain error falls
    and its time grows with the photon count, so the plain tracer needs more
    photons than the largest measured run whose error is still above `target`
    (lower bound: that run's time over the denoised time) and no more than the
    smallest run at or below it (upper bound). `extra_ms` is added to each
    plain time (the direct-beam solve in the like-for-like comparison).
    Returns [low, high]; a side without such a run is None."""
    runs = sorted(zip(plain_ppc, rmse, ms))
    above = [m for _, e, m in runs if e > target]
    below = [m for _, e, m in runs if e <= target]
    low = (above[-1] + extra_ms) / t_denoised if above else None
    high = (below[0] + extra_ms) / t_denoised if below else None
    return [low, high]


def plain_ppc_to_match(plain_ppc, rmse, target, truth_ppc=None):
    """Photons/column at which the plain tracer's RMSE reaches `target`.

    Errors are measured against a truth run of `truth_ppc` photons/column,
    which has Monte Carlo noise of its own, independent of the run under
    test. The plain tracer's noise falls as N^-1/2 (Sec. 3.2), so a plain run
    of p photons/column measures
        rmse^2 = a^2 (1/p + 1/truth_ppc),
    and a target measured the same way is reached at
        1/N = target^2 / a^2 - 1/truth_ppc.
    a is the geometric mean of rmse / sqrt(1/p + 1/truth_ppc) over the runs.
    truth_ppc None drops the truth term (a noise-free truth). A target at or
    below the truth's own noise floor returns inf: no plain run can be shown
    to reach it against that truth."""
    it = 0.0 if truth_ppc is None else 1.0 / truth_ppc
    a = float(np.exp(np.mean([math.log(e / math.sqrt(1.0 / p + it)) for p, e in zip(plain_ppc, rmse)])))
    inv_n = (target / a) ** 2 - it
    return math.inf if inv_n <= 0.0 else 1.0 / inv_n


def torch_rms(a, b):
    """RMS difference of two device tensors."""
    return ((a - b) ** 2).mean().sqrt().item()


def _errors(fields, truth, hf, shape):
    nz, ny, nx = shape
    a = fields[0].cpu().numpy().reshape(nz, ny, nx)
    at = truth[0].cpu().numpy().reshape(nz, ny, nx)
    ghi = (fields[1] + fields[2]).cpu().numpy()
    ght = (truth[1] + truth[2]).cpu().numpy()
    hr = (a - at) * hf[:, None, None]
    return float(np.sqrt(((ghi - ght) ** 2).mean())), float(np.sqrt((hr ** 2).mean()))


def evaluate(net, seeds, shape, lo_ppc=4, plain_ppc=(4, 16, 64, 256, 1024, 4096, 16384), truth_ppc=65536, workers=8,
             repeats=3, spectral=False, direct_nsub=8, direct_features=False, exact_direct=True):
    """Time-to-RMSE of denoised low-photon runs against the plain tracer.

    For each held-out scene: a truth run at `truth_ppc`, plain runs at each
    of `plain_ppc` (RMSE of GHI and heating rate, and wall time of the trace
    plus field read-out, CUDA events), and the denoised run (trace at `lo_ppc`
    + packing + network + unpacking). The plain RMSE is fitted as a N^-1/2
    (Sec. 3.2) to find the photon count that reaches the denoised RMSE; the
    plain time at that count is interpolated between the measured runs
    (plain_time_at), and the speed-up is that time over the denoised wall
    time. Every RMSE is measured against the truth run, whose own noise is
    modelled in the match (plain_ppc_to_match with truth_ppc).
    `speedup_bracket` bounds the same speed-ups with no model at all.

    Surface direct irradiance of the denoised product (one quadrature point,
    `exact_direct`): the expected value from the pixel-mean Beer-Lambert
    transmittance (`direct_nsub`^2 points per column, nn_direct_surface),
    included in the timed region (on a second stream, beside the trace);
    the network supplies absorption and diffuse irradiance. Otherwise all
    three come from the network. The GHI speed-up (speedup_ghi) then compares
    like with like: the plain tracer is given the same exact direct beam, so
    the two GHI errors differ only in the diffuse part, and the plain time
    includes the direct solve. `surface` reports direct and diffuse RMS
    errors separately, the network's own surface-direct error, and the GHI
    speed-up against a plain tracer that traces its direct part.
    """
    torch = _torch()
    nz, ny, nx = shape
    scs = make_scenes(seeds, nx, ny, nz, workers)
    ft = FieldTracer(shape, spectral=spectral, direct_features=direct_features)
    hf = heating_factor(nz, ft.dz)
    stream = torch.cuda.current_stream()
    acc = {p: [0.0, 0.0, 0.0] for p in plain_ppc}
    den = [0.0, 0.0, 0.0]
    noisy = [0.0, 0.0]
    hybrid = exact_direct and not spectral
    dms_sum = 0.0
    comp = {}                                # direct and diffuse RMS errors^2, summed over scenes

    def add(key, a, b):
        comp[key] = comp.get(key, 0.0) + torch_rms(a, b) ** 2

    def timed(fn):
        best = None
        res = None
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = fn()
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return res, best

    side = torch.cuda.Stream()
    for seed, sc in zip(seeds, scs):
        sza = SZAS[seed % 3]
        ft.load(sc)
        truth = tuple(t.clone() for t in ft.trace(sza, truth_ppc, 7 * seed + 1))
        if hybrid:
            sdx, dms = timed(lambda: ft.direct_surface(sza, direct_nsub))
            dms_sum += dms
            add("exact_dir", sdx, truth[1])
        for p in plain_ppc:
            f, ms = timed(lambda: ft.trace(sza, p, 7 * seed + 2 + p))
            e1, e2 = _errors(f, truth, hf, shape)
            acc[p][0] += e1 ** 2; acc[p][1] += e2 ** 2; acc[p][2] += ms
            if hybrid:
                add("plain%d_dir" % p, f[1], truth[1])
                add("plain%d_dif" % p, f[2], truth[2])

        def run():
            if hybrid:
                # the direct-beam solve needs only the optics: it runs on a
                # second stream while the trace's last long histories finish
                side.wait_stream(stream)
                sdx = ft.direct_surface(sza, direct_nsub, stream=side)
            lo = ft.trace(sza, lo_ppc, 7 * seed + 3)
            fnet = denoise(net, ft.pack(lo, sza))
            if hybrid:
                stream.wait_stream(side)
                sdx.record_stream(stream)
                return (fnet[0], sdx, fnet[2]), fnet, lo
            return fnet, fnet, lo
        (fd, fnet, lo), ms = timed(run)
        e1, e2 = _errors(fd, truth, hf, shape)
        den[0] += e1 ** 2; den[1] += e2 ** 2; den[2] += ms
        n1, n2 = _errors(lo, truth, hf, shape)
        noisy[0] += n1 ** 2; noisy[1] += n2 ** 2
        if hybrid:
            add("network_ghi", fnet[1] + fnet[2], truth[1] + truth[2])
            add("network_dir", fnet[1], truth[1])
            add("den_dif", fd[2], truth[2])
            add("noisy_dir", lo[1], truth[1])
            add("noisy_dif", lo[2], truth[2])
    ft.close()
    n = len(seeds)
    plain = {p: {"rmse_ghi": math.sqrt(v[0] / n), "rmse_hr": math.sqrt(v[1] / n), "ms": v[2] / n}
             for p, v in acc.items()}
    res = {"shape": shape, "scenes": n, "truth_ppc": truth_ppc, "spectral": spectral,
           "quadrature_points": len(ft.gflux) if spectral else 1, "plain": plain,
           "denoised": {"ppc": lo_ppc, "rmse_ghi": math.sqrt(den[0] / n), "rmse_hr": math.sqrt(den[1] / n),
                        "ms": den[2] / n},
           "noisy_input": {"rmse_ghi": math.sqrt(noisy[0] / n), "rmse_hr": math.sqrt(noisy[1] / n)}}
    # plain tracer: rmse^2 = a^2 (1/ppc + 1/truth_ppc); its time at a photon
    # count interpolated between the measured runs (the least-squares line is
    # reported for reference only: the large runs pull it away from the
    # small ones)
    t0, t1 = plain_time_fit(plain_ppc, [plain[p]["ms"] for p in plain_ppc])
    res["plain_time_fit_ms"] = {"t0": t0, "per_ppc": t1}
    plain_ms = [plain[p]["ms"] for p in plain_ppc]

    def t_plain(n):
        return plain_time_at(plain_ppc, plain_ms, n)
    res["fit"] = ("plain rmse^2 = a^2 (1/ppc + 1/truth_ppc), a the geometric mean over the plain runs; "
                  "plain time interpolated linearly between the measured runs, extended beyond the largest "
                  "at the rate of the last two")
    for key in ("rmse_ghi", "rmse_hr"):
        ppc_match = plain_ppc_to_match(plain_ppc, [plain[p][key] for p in plain_ppc], res["denoised"][key],
                                       truth_ppc)
        t_match = t_plain(ppc_match)
        name = key.split("_")[1]
        res["plain_ppc_to_match_" + name] = ppc_match
        res["plain_ms_to_match_" + name] = t_match
        res["speedup_" + name] = t_match / res["denoised"]["ms"]
        res.setdefault("speedup_bracket", {})[name] = speedup_bracket(
            plain_ppc, [plain[p][key] for p in plain_ppc], [plain[p]["ms"] for p in plain_ppc],
            res["denoised"][key], res["denoised"]["ms"])
    res["surface"] = {"direct": "network"}
    if hybrid:
        res["surface"] = {"direct": "exact pixel-mean Beer-Lambert, %d x %d points per column" % (direct_nsub,
                                                                                                  direct_nsub),
                          "direct_solve_ms_alone": dms_sum / n,
                          "rmse": {k: math.sqrt(v / n) for k, v in comp.items()}}
        # the plain tracer tracing its own direct part: GHI errors as measured
        res["surface"]["speedup_ghi_vs_plain_traced_direct"] = res["speedup_ghi"]
        res["surface"]["plain_ppc_to_match_ghi_traced_direct"] = res["plain_ppc_to_match_ghi"]
        # Like for like, the headline: the plain tracer given the same exact
        # direct beam. Both GHI errors then share the direct term and differ
        # only in the diffuse part; the plain time includes the direct solve.
        p_dif = plain_ppc_to_match(plain_ppc, [math.sqrt(comp["plain%d_dif" % p] / n) for p in plain_ppc],
                                   math.sqrt(comp["den_dif"] / n), truth_ppc)
        res["plain_ppc_to_match_ghi"] = p_dif
        res["plain_ms_to_match_ghi"] = t_plain(p_dif) + dms_sum / n
        res["speedup_ghi"] = res["plain_ms_to_match_ghi"] / res["denoised"]["ms"]
        res["surface"]["speedup_ghi_vs_plain_exact_direct"] = res["speedup_ghi"]
        res["speedup_bracket"]["ghi"] = speedup_bracket(
            plain_ppc, [math.sqrt(comp["plain%d_dif" % p] / n) for p in plain_ppc],
            [plain[p]["ms"] for p in plain_ppc], math.sqrt(comp["den_dif"] / n), res["denoised"]["ms"],
            extra_ms=dms_sum / n)
        # the network's own surface-direct estimate, for comparison
        p_net = plain_ppc_to_match(plain_ppc, [plain[p]["rmse_ghi"] for p in plain_ppc],
                                   math.sqrt(comp["network_ghi"] / n), truth_ppc)
        res["surface"]["network_only_speedup_ghi"] = t_plain(p_net) / res["denoised"]["ms"]
    return res


def main(argv=None):
    """Train on seeded scenes and report time-to-RMSE on held-out scenes (JSON)."""
    import argparse
    import json
    p = argparse.ArgumentParser(description="train and evaluate the 3D U-Net denoiser")
    p.add_argument("--train", type=int, default=512, help="training scenes (seeds 1000...)")
    p.add_argument("--eval", type=int, default=64, help="held-out scenes (seeds after the training ones)")
    p.add_argument("--epochs", type=int, default=32)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--warmup", type=float, default=0.05, help="fraction of the steps with a linear learning-rate ramp")
    p.add_argument("--seed", type=int, default=0, help="order of the training scenes")
    p.add_argument("--shape", type=int, nargs=3, default=(128, 128, 128), help="nz ny nx")
    p.add_argument("--truth-ppc", type=int, default=65536)
    p.add_argument("--hi-ppc", type=int, default=1024, help="photons/column of the training targets")
    p.add_argument("--lo-ppc", type=int, default=4, help="photons/column of the network's traced input")
    p.add_argument("--plain-ppc", type=int, nargs="+", default=(4, 16, 64, 256, 1024, 4096, 16384))
    p.add_argument("--spectral", action="store_true",
                   help="broadband fields: all quadrature points of the g-point table in one batched launch")
    p.add_argument("--workers", type=int, default=16)
    p.add_argument("--direct-features", action="store_true",
                   help="input channels 6, 7: deterministic direct-beam transmittance (voxel, pixel-mean surface)")
    p.add_argument("--direct-loss", action="store_true",
                   help="train on the surface-direct channel too and take the network's surface direct "
                        "(default: the exact direct beam, and no direct term in the loss)")
    p.add_argument("--out", default=None, help="write the result JSON here")
    a = p.parse_args(argv)
    shape = tuple(a.shape)
    t0 = time.time()
    pairs = make_pairs(list(range(1000, 1000 + a.train)), shape, lo_ppc=a.lo_ppc, hi_ppc=a.hi_ppc, workers=a.workers,
                       spectral=a.spectral, direct_features=a.direct_features)
    t_pairs = time.time() - t0
    net = UNet(seed=0)
    chw = channel_weights(pairs, direct=a.direct_loss)
    t0 = time.time()
    losses = train(net, pairs, epochs=a.epochs, lr=a.lr, chw=chw, log=lambda s: print(s, flush=True),
                   warmup=a.warmup, seed=a.seed)
    t_train = time.time() - t0
    del pairs
    res = evaluate(net, list(range(1000 + a.train, 1000 + a.train + a.eval)), shape, lo_ppc=a.lo_ppc,
                   truth_ppc=a.truth_ppc,
                   workers=a.workers, plain_ppc=tuple(a.plain_ppc), spectral=a.spectral,
                   direct_features=a.direct_features, exact_direct=not a.direct_loss)
    res.update({"train_scenes": a.train, "epochs": a.epochs, "lo_ppc": a.lo_ppc, "hi_ppc": a.hi_ppc, "warmup": a.warmup, "seed": a.seed,
                "direct_features": a.direct_features, "direct_loss": a.direct_loss, "guards": net.train_log, "pairs_s": t_pairs, "train_s": t_train,
                "loss_first": losses[0][1], "loss_last": losses[-1][1], "params": net.n_params(),
                "forward_gflop": net.flops(shape) / 1e9})
    print(json.dumps(res), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    return res


if __name__ == "__main__":
    main()
