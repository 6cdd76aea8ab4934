"""Overlapped steps of the tracer: a ring of handles, and a host pipeline.

A step (new optics, accelerator build, one trace, the fields read out) ends
with a latency tail: when the photon queue is empty, a few long histories in
thick cloud run on nearly idle SMs for about a quarter of the launch. Handles
are independent, so `StepRing` gives each of two handles its own stream and
alternates steps between them: the next step's optics, accelerator and
transport start on the SMs that the previous step's finished blocks release.

A host-side caller (for instance an atmospheric model stepping on the CPU)
hands the tracer new optics every step and reads the fields back. Done one
call after the other, the 170 MB of input copies and 140 MB of output copies of
the 256 x 256 x 128 scene add a quarter to every step. `HostPipeline` overlaps
them with the transport: while step k traces, step k+1's optics travel to the
device on one copy stream and step k-1's fields travel back on another,
through two sets of device buffers, and with two handles the steps' transport
overlaps as in `StepRing`. Every computation still runs through the library's
C calls (rt_set_optics, rt_set_surface, rt_build_accel, rt_trace_range,
rt_fields, rt_heating_rate) on device buffers; torch provides the buffers,
streams and events.
"""
from __future__ import annotations

from . import rt

OUT_KEYS = ("abs3d", "hr", "sfc_dir", "sfc_dif", "toa_up")


def _tracers(tracers):
    ts = [tracers] if isinstance(tracers, rt.Tracer) else list(tracers)
    if not ts:
        raise ValueError("no tracer handles")
    g = (ts[0].nx, ts[0].ny, ts[0].nz)
    if any((t.nx, t.ny, t.nz) != g for t in ts):
        raise ValueError("the handles of one ring must have the same grid")
    return ts


class StepRing:
    """Steps on device-resident inputs, alternating between the given Tracer
    handles (one stream each; two are enough to cover the tail). Step k runs
    on handle k mod len(tracers) and writes that handle's own output buffers,
    which stay valid until the handle's next step is submitted. The handles
    keep the ring's streams: give them another one (Tracer.set_stream) before
    using them outside the ring."""

    def __init__(self, tracers, coarse=(0, 0, 0)):
        import torch
        self.torch = torch
        self.ts = _tracers(tracers)
        self.coarse = tuple(coarse)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=dev) for _ in self.ts]
        for t, s in zip(self.ts, self.streams):
            t.set_stream(s)
        n3, n2 = self.ts[0].ncell, self.ts[0].ncol
        # each handle's outputs belong to its stream in torch's allocator, so
        # their memory is not handed out again before that stream's work on
        # them is done
        self.out = []
        for s in self.streams:
            with torch.cuda.stream(s):
                self.out.append({k: torch.empty(n3 if k in ("abs3d", "hr") else n2, dtype=torch.float64,
                                                device=dev) for k in OUT_KEYS})
        self.k = 0

    def submit(self, fields, albedo, sza, az, flux, photons, seed, photon_begin=0, photons_total=None,
               events=None, after=None):
        """Enqueue one step on the next handle: the five optics fields and the
        albedo (device tensors, read by rt_set_optics / rt_set_surface), an
        accelerator build, `photons` photons from id `photon_begin` of a run of
        `photons_total`, and the fields. `events` (two CUDA events) are
        recorded around the transport launch; `after(stream, out)` runs on the
        handle's stream once the fields are written. Inputs written on another
        stream must be ordered first (`wait_on`). Returns (handle index, output
        dict)."""
        torch = self.torch
        j = self.k % len(self.ts)
        t, st, o = self.ts[j], self.streams[j], self.out[j]
        t.set_optics(*fields)
        t.set_surface(albedo)
        t.build_accel(*self.coarse)
        t.reset()
        if events is not None:
            events[0].record(st)
        rt.rt_trace_range(t.h, sza, az, flux, photon_begin, photons, photons_total or photons, seed)
        if events is not None:
            events[1].record(st)
        rt.rt_fields(t.h, t.ncell, t.ncol, o["abs3d"], o["sfc_dir"], o["sfc_dif"], o["toa_up"])
        rt.rt_heating_rate(t.h, t.ncell, o["hr"], 0)
        if after is not None:
            with torch.cuda.stream(st):
                after(st, o)
        self.k += 1
        return j, o

    def wait_on(self, stream):
        """Make every handle's stream wait for the work queued so far on `stream`."""
        for s in self.streams:
            s.wait_stream(stream)

    def join(self, stream):
        """Make `stream` wait for every handle's queued work."""
        for s in self.streams:
            stream.wait_stream(s)

    def synchronize(self):
        for t in self.ts:
            t.synchronize()


class HostPipeline:
    """Pipelined steps of one Tracer, or alternating between several (one
    stream each). Host buffers must be pinned (torch tensors with
    pin_memory()) for the copies to overlap. The device buffers serve several
    streams: call synchronize() before dropping the pipeline, so that no copy
    or kernel still uses them when torch's allocator takes them back."""

    def __init__(self, tracers, coarse=(0, 0, 0)):
        import torch
        self.torch = torch
        self.ts = _tracers(tracers)
        self.t = self.ts[0]
        self.coarse = tuple(coarse)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.compute = [torch.cuda.Stream(device=dev) for _ in self.ts]
        # separate copy streams in and out: an input copy queued behind the
        # previous step's output copy would wait for that step's transport
        self.copy_in = torch.cuda.Stream(device=dev)
        self.copy_out = torch.cuda.Stream(device=dev)
        for t, s in zip(self.ts, self.compute):
            t.set_stream(s)
        # device buffer sets: two, or one per handle when there are more
        self.nbuf = nb = max(2, len(self.ts))
        if nb % len(self.ts):
            raise ValueError("use 1, 2 or more handles that divide the buffer count")
        n3, n2 = self.t.ncell, self.t.ncol
        f32, f64 = torch.float32, torch.float64
        self.d_in = [[torch.empty(n3, dtype=f32, device=dev) for _ in range(5)] for _ in range(nb)]
        self.d_alb = [torch.empty(n2, dtype=f32, device=dev) for _ in range(nb)]
        self.d_out = [{k: torch.empty(n3 if k in ("abs3d", "hr") else n2, dtype=f64, device=dev) for k in OUT_KEYS}
                      for _ in range(nb)]
        ev = lambda: [torch.cuda.Event() for _ in range(nb)]   # noqa: E731
        self.in_ready, self.in_free = ev(), ev()
        self.out_ready, self.out_free = ev(), ev()
        self.k = 0

    def submit(self, fields, albedo, sza, az, flux, photons, seed, out, photon_begin=0, photons_total=None):
        """Enqueue one step: copy the five optics fields and the albedo (pinned
        host tensors) in, trace `photons` photons, and copy the fields into
        `out` (dict of pinned host tensors keyed abs3d, hr, sfc_dir, sfc_dif,
        toa_up). `out` is complete after `synchronize()`."""
        torch = self.torch
        nb = self.nbuf
        b = self.k % nb
        j = self.k % len(self.ts)
        t, comp = self.ts[j], self.compute[j]
        with torch.cuda.stream(self.copy_in):
            if self.k >= nb:
                self.copy_in.wait_event(self.in_free[b])
            for d, h in zip(self.d_in[b], fields):
                d.copy_(h.reshape(-1), non_blocking=True)
            self.d_alb[b].copy_(albedo.reshape(-1), non_blocking=True)
            self.in_ready[b].record(self.copy_in)
        comp.wait_event(self.in_ready[b])
        t.set_optics(*self.d_in[b])
        t.set_surface(self.d_alb[b])
        self.in_free[b].record(comp)
        t.build_accel(*self.coarse)
        t.reset()
        total = photons_total or photons
        rt.rt_trace_range(t.h, sza, az, flux, photon_begin, photons, total, seed)
        if self.k >= nb:
            comp.wait_event(self.out_free[b])
        o = self.d_out[b]
        rt.rt_fields(t.h, t.ncell, t.ncol, o["abs3d"], o["sfc_dir"], o["sfc_dif"], o["toa_up"])
        rt.rt_heating_rate(t.h, t.ncell, o["hr"], 0)
        self.out_ready[b].record(comp)
        with torch.cuda.stream(self.copy_out):
            self.copy_out.wait_event(self.out_ready[b])
            for k in OUT_KEYS:
                out[k].view(-1).copy_(o[k], non_blocking=True)
            self.out_free[b].record(self.copy_out)
        self.k += 1

    def synchronize(self):
        self.copy_in.synchronize()
        for s in self.compute:
            s.synchronize()
        self.copy_out.synchronize()
        for t in self.ts:
            t.synchronize()
