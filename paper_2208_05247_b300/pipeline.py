"""Double-buffered host <-> device pipeline for repeated radiation calls.

A host-side caller (for instance an atmospheric model stepping on the CPU)
hands the tracer new optics every step and reads the fields back. Done one
call after the other, the 170 MB of input copies and 140 MB of output copies of
the 256 x 256 x 128 scene add a quarter to every step. `HostPipeline` overlaps
them with the transport: while step k traces on the tracer's stream, step
k+1's optics travel to the device on one copy stream and step k-1's fields
travel back on another, through two sets of device buffers. Every computation still
runs through the library's C calls (rt_set_optics, rt_set_surface,
rt_build_accel, rt_trace_range, rt_fields, rt_heating_rate) on device
buffers; torch provides the buffers, streams and events.
"""
from __future__ import annotations

from . import rt

OUT_KEYS = ("abs3d", "hr", "sfc_dir", "sfc_dif", "toa_up")


class HostPipeline:
    """Pipelined steps of one Tracer. Host buffers must be pinned (torch
    tensors with pin_memory()) for the copies to overlap."""

    def __init__(self, tracer: rt.Tracer, coarse=(0, 0, 0)):
        import torch
        self.torch = torch
        self.t = tracer
        self.coarse = tuple(coarse)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.compute = torch.cuda.Stream(device=dev)
        # separate copy streams in and out: an input copy queued behind the
        # previous step's output copy would wait for that step's transport
        self.copy_in = torch.cuda.Stream(device=dev)
        self.copy_out = torch.cuda.Stream(device=dev)
        tracer.set_stream(self.compute)
        n3, n2 = tracer.ncell, tracer.ncol
        f32, f64 = torch.float32, torch.float64
        self.d_in = [[torch.empty(n3, dtype=f32, device=dev) for _ in range(5)] for _ in range(2)]
        self.d_alb = [torch.empty(n2, dtype=f32, device=dev) for _ in range(2)]
        self.d_out = [{k: torch.empty(n3 if k in ("abs3d", "hr") else n2, dtype=f64, device=dev) for k in OUT_KEYS}
                      for _ in range(2)]
        ev = lambda: torch.cuda.Event()   # noqa: E731
        self.in_ready, self.in_free = [ev(), ev()], [ev(), ev()]
        self.out_ready, self.out_free = [ev(), ev()], [ev(), ev()]
        self.k = 0

    def submit(self, fields, albedo, sza, az, flux, photons, seed, out, photon_begin=0, photons_total=None):
        """Enqueue one step: copy the five optics fields and the albedo (pinned
        host tensors) in, trace `photons` photons, and copy the fields into
        `out` (dict of pinned host tensors keyed abs3d, hr, sfc_dir, sfc_dif,
        toa_up). `out` is complete after `synchronize()`."""
        torch = self.torch
        b = self.k & 1
        with torch.cuda.stream(self.copy_in):
            if self.k >= 2:
                self.copy_in.wait_event(self.in_free[b])
            for d, h in zip(self.d_in[b], fields):
                d.copy_(h.reshape(-1), non_blocking=True)
            self.d_alb[b].copy_(albedo.reshape(-1), non_blocking=True)
            self.in_ready[b].record(self.copy_in)
        self.compute.wait_event(self.in_ready[b])
        t = self.t
        t.set_optics(*self.d_in[b])
        t.set_surface(self.d_alb[b])
        self.in_free[b].record(self.compute)
        t.build_accel(*self.coarse)
        t.reset()
        total = photons_total or photons
        rt.rt_trace_range(t.h, sza, az, flux, photon_begin, photons, total, seed)
        if self.k >= 2:
            self.compute.wait_event(self.out_free[b])
        o = self.d_out[b]
        rt.rt_fields(t.h, t.ncell, t.ncol, o["abs3d"], o["sfc_dir"], o["sfc_dif"], o["toa_up"])
        rt.rt_heating_rate(t.h, t.ncell, o["hr"], 0)
        self.out_ready[b].record(self.compute)
        with torch.cuda.stream(self.copy_out):
            self.copy_out.wait_event(self.out_ready[b])
            for k in OUT_KEYS:
                out[k].view(-1).copy_(o[k], non_blocking=True)
            self.out_free[b].record(self.copy_out)
        self.k += 1

    def synchronize(self):
        self.copy_in.synchronize()
        self.compute.synchronize()
        self.copy_out.synchronize()
        self.t.synchronize()
