#!/usr/bin/env python
"""Benchmark of the B300 shortwave Monte Carlo tracer.

Workload: the LES-like cumulus scene (256 x 256 x 128 cells, dx = dy = 50 m,
dz = 25 m, seeded sum of 400 Gaussian blobs, 20 % cloud cover), solar zenith
30 deg, 256 photons per column (16.8 M photons per step), TOA flux 1000 W m^-2.

One step is the whole hot path through the C ABI, with inputs resident in HBM:
optics derivation + validation, surface check, majorant grid, tally reset,
the persistent transport kernel, and the FP64 output fields (3D absorption,
surface direct/diffuse, top upward flux, heating rate) into device buffers.

Prints one JSON line. `value` is majorant collision events per second over
the timed steps, which alternate between two tracer handles on two streams so
that one step's transport tail overlaps the next step (`--streams 1`: one
after the other, also timed as `serial_ms_per_step`); CUDA events on the
default stream, which waits for both. `e2e` is the same metric through the C
ABI with host buffers (host->device inputs and device->host outputs inside the
timed region). `roofline` uses the transport kernel's own CUDA-event duration
in the single-stream loop, where one launch has the GPU to itself. `cpu_baseline` times the FP64 CPU oracle on a bounded
sample of the same scene.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon collision events/s & wall time to target RMS GHI/heating error, denoised vs plain"
UNIT = "events/s"
SZA, AZ, F0 = 30.0, 0.0, 1000.0
SEED = 20220926
COARSE = (2, 2, 2)
# Algorithmic bytes of the transport kernel: 16 B optics record + 16 B FP64
# tally read-modify-write per majorant event, 4 B majorant box word per walk
# step (the "crossings" counter).
BYTES_PER_EVENT, BYTES_PER_CROSSING = 32, 4
# derive, albedo check, two status-word stores (the optics and albedo checks
# read back), majorant, majorant boxes (init + 4 levels of 3 axis dilations and
# a selection), column keys + column order (launch order), transport, 4 field
# sums, heating rate
KERNELS_PER_STEP = 30
PROFILE = os.path.join(ROOT, "profiles", "trace_kernel_cumulus256.md")


def parse():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--ppc", type=int, default=256, help="photons per column per step")
    p.add_argument("--sza", type=float, default=SZA)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-ppc", type=int, default=16)
    p.add_argument("--no-denoise", action="store_true", help="skip the denoised-vs-plain time-to-RMSE leg")
    p.add_argument("--no-coupled", action="store_true", help="skip the graph-replay coupled-step leg")
    p.add_argument("--no-birth", action="store_true", help="skip the Sobol-vs-Philox start position leg")
    p.add_argument("--no-batched", action="store_true", help="skip the batched multi-scene workload leg")
    p.add_argument("--no-sweep", action="store_true", help="skip the sun-angle x photons-per-column sweep")
    p.add_argument("--denoise-train", type=int, default=512, help="training scenes of the denoiser leg")
    p.add_argument("--denoise-eval", type=int, default=64, help="held-out scenes of the denoiser leg")
    p.add_argument("--no-l2-probe", action="store_true", help="skip the L2 read-bandwidth probe")
    p.add_argument("--denoise-epochs", type=int, default=32, help="training epochs of the denoiser leg")
    p.add_argument("--denoise-lo-ppc", type=int, default=4,
                   help="photons/column of the denoiser's traced input (4: the configured workload)")
    p.add_argument("--streams", type=int, default=2,
                   help="tracer handles (one stream each) that the timed steps alternate between; 1 = one after "
                        "the other")
    p.add_argument("--reduce-fields", action="store_true",
                   help="N>1: sum the ranks' output fields every step (NCCL all-reduce) into one combined field")
    p.add_argument("--no-autotune", action="store_true",
                   help="use the default launch parameters and the --coarse grid")
    p.add_argument("--coarse", type=int, nargs=3, default=None,
                   help="coarse grid factors; implies --no-autotune")
    p.add_argument("--launch", type=int, nargs=3, default=None, metavar=("READY", "INNER", "CHUNK"),
                   help="ready_threshold, max_inner and refill_chunk of the transport launch "
                        "(with --coarse: the autotuner's choice without rerunning it)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def workload_config(args, world, coarse=COARSE):
    return {"workload": f"cumulus 256x256x128 (dx=dy=50 m, dz=25 m, 400 blobs, 20% cloud), "
                        f"sza {args.sza:g}, {args.ppc} photons/column, {args.ppc * 65536} photons per GPU "
                        f"per step, coarse grid {coarse[0]}x{coarse[1]}x{coarse[2]}",
            "photons_per_step": args.ppc * 65536 * world,
            "l2": "inputs larger than L2: 168 MB optics + 134 MB derived records + 135 MB FP64 tallies",
            "parallelism": f"photon ranges, {world} rank(s), no data-path collective"}


# ---- clocks during the timed region ---------------------------------------------------

class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            self.sel = str(device_index)

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.sel, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) == 7:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[3:]) if v.lower() == "active"})
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("rt_device.cuh", "rt_kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2208_05247_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it matches the source."""
    try:
        kv = {}
        for line in open(PROFILE):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_hash") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


# ---- CPU oracle (baseline and reference arm) ------------------------------------------

def oracle_sample(scene, ppc: int, seed: int):
    import oracle
    n = ppc * scene.ncol
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.trace(scene, SZA, AZ, F0, n, seed, nthreads=cores)
    dt = time.perf_counter() - t0
    return r.totals, dt, cores


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2208_05247_b300 import scenes
    scene = scenes.cumulus_scene(seed=1)
    ppc = 1
    for w in range(args.warmup):
        oracle_sample(scene, ppc, SEED + w)
    coll, photons, secs, cores = 0, 0, 0.0, 1
    for k in range(args.steps):
        tot, dt, cores = oracle_sample(scene, ppc, SEED + 100 + k)
        coll += tot["collisions"]
        photons += tot["photons"]
        secs += dt
    value = coll / secs
    sample = (f"each step {ppc} photon/column ({ppc * scene.ncol} photons) of the benchmark scene; "
              f"oracle collisions (analog: every collision is real)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "photons_per_s": photons / secs,
            "config": dict(workload_config(args, 1),
                           sample=f"bounded sample: each step traces {ppc} photon/column ({ppc * scene.ncol} "
                                  f"photons) of this workload with the FP64 analog oracle, not "
                                  f"{args.ppc} photons/column",
                           photons_per_step_traced=ppc * scene.ncol),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "photons_per_s": photons / secs,
                             "note": "events are the oracle's real (analog) collisions; the GPU arm counts "
                                     "majorant events, null collisions included, so photons_per_s is the "
                                     "like-for-like rate"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "photons_per_s": photons / secs}}
    print(json.dumps(line), flush=True)


# ---- the full config-1 grid: sun angles x photons per column ------------------------------

def sweep_leg(t, coarse):
    """Transport on the benchmark scene at every sun angle and photon count of
    the workload (SZA 0, 30, 60 x 1, 4, 16, 64, 256 photons/column): CUDA-event
    time of one trace (best of 3 after a warm-up), photons/s and majorant
    events/s. The tracer keeps the bench's launch configuration."""
    import torch
    stream = torch.cuda.current_stream()
    ncol = t.nx * t.ny
    rows = []
    for sza in (0.0, 30.0, 60.0):
        for ppc in (1, 4, 16, 64, 256):
            best = None
            for r in range(4):
                t.reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                t.trace(sza, AZ, F0, ppc * ncol, SEED + 50 + r)
                b.record(stream)
                b.synchronize()
                if r:
                    ms = a.elapsed_time(b)
                    best = ms if best is None else min(best, ms)
            st = t.stats()
            rows.append({"sza": sza, "ppc": ppc, "ms": best, "photons_per_s": ppc * ncol / (best / 1e3),
                         "events_per_s": st["events"] / (best / 1e3), "events_per_photon": st["events"] / (ppc * ncol),
                         "max_events_photon": st["max_events_photon"]})
    return {"workload": "cumulus 256x256x128, coarse grid %dx%dx%d, one trace per point" % tuple(coarse),
            "rows": rows}


# ---- denoised vs plain: wall time to a target RMS error ----------------------------------

def denoise_leg(args):
    """Train the 3D U-Net on tracer pairs (4 vs 1024 photons/column of one
    quadrature point, 128^3 cumulus scenes; --denoise-lo-ppc changes the 4)
    and time denoised runs against the plain tracer at matched RMS error of
    GHI and heating rate on held-out scenes."""
    from paper_2208_05247_b300 import denoise
    shape = (128, 128, 128)
    t0 = time.time()
    pairs = denoise.make_pairs(list(range(1000, 1000 + args.denoise_train)), shape, lo_ppc=args.denoise_lo_ppc,
                               workers=os.cpu_count() or 8)
    t_pairs = time.time() - t0
    net = denoise.UNet(seed=0)
    t0 = time.time()
    # no surface-direct term in the loss: the product takes the exact direct beam
    losses = denoise.train(net, pairs, epochs=args.denoise_epochs, lr=1e-3,
                           chw=denoise.channel_weights(pairs, direct=False))
    t_train = time.time() - t0
    del pairs
    res = denoise.evaluate(net, list(range(1512, 1512 + args.denoise_eval)), shape, lo_ppc=args.denoise_lo_ppc,
                           truth_ppc=65536, workers=os.cpu_count() or 8)
    return {"workload": "one quadrature point on cumulus 128x128x128 (dx=dy=50 m, dz=25 m), sza 0/30/60, "
                        f"{args.denoise_eval} held-out scenes (seeds 1512-{1511 + args.denoise_eval}), "
                        f"truth 65536 photons/column, plain runs 4-16384 photons/column, traced input "
                        f"{args.denoise_lo_ppc} photons/column",
            "fit": res["fit"], "plain_time_fit_ms": res["plain_time_fit_ms"],
            "training": {"scenes": args.denoise_train, "epochs": args.denoise_epochs, "pairs_s": t_pairs,
                         "train_s": t_train, "weights": "moving average over the last tenth of the steps",
                         "schedule": "Adam, linear warmup over 5 % of the steps, cosine decay 1e-3 to 1e-4",
                         "guards": getattr(net, "train_log", None),
                         "loss_first": losses[0][1], "loss_last": losses[-1][1]},
            "plain": res["plain"], "denoised": res["denoised"], "noisy_input": res["noisy_input"],
            "plain_ppc_to_match": {"ghi": res["plain_ppc_to_match_ghi"], "hr": res["plain_ppc_to_match_hr"]},
            "speedup": {"ghi": res["speedup_ghi"], "hr": res["speedup_hr"],
                        "ghi_basis": "like for like: the plain tracer gets the same exact direct beam "
                                     "(its time includes the direct solve), so the GHI errors differ only in "
                                     "the diffuse part"},
            "speedup_bracket": dict(res["speedup_bracket"],
                                    note="no fit: the measured plain runs either side of the denoised error "
                                         "(lower, upper; None where no run lies on that side)"),
            "surface": res.get("surface"),
            "network": {"params": net.n_params(), "forward_gflop": net.flops(shape) / 1e9}}


# ---- coupled-model step: graph replay vs the ordinary calls ------------------------------

def coupled_step_leg(t, d_in, d_alb, d_out, photons, eager_ms, eager_events, steps):
    """Time the same step recorded as one CUDA graph (rt_step) with inputs
    bound in place: no host synchronisation inside the step."""
    import torch
    from paper_2208_05247_b300 import rt
    stream = torch.cuda.current_stream()
    step = rt.rt_step_create(t.h, t.ncell, t.ncol, d_in, photons, albedo=d_alb, **d_out)
    try:
        for _ in range(3):
            rt.rt_step_launch(step, SZA, AZ, F0, 0.0, SEED)
        rt.rt_synchronize(t.h)
        assert t.stats()["events"] == eager_events, "graph replay traced different histories"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            rt.rt_step_launch(step, SZA, AZ, F0, 0.0, SEED)
        e1.record(stream)
        rt.rt_synchronize(t.h)
        ms = e0.elapsed_time(e1) / steps
        # the launch overhead alone: a step of one photon per column
    finally:
        rt.rt_step_destroy(step)
    return {"graph_ms_per_step": ms, "eager_ms_per_step": eager_ms, "steps": steps,
            "host_syncs_per_step": {"graph": 0, "eager": 2},
            "note": "same kernels and arguments; the graph replays optics derivation, majorant, reset, "
                    "transport and outputs from device buffers updated in place (Sec. 2.2 coupling)"}


# ---- scrambled Sobol vs Philox start positions: error at equal photons ---------------------

def birth_leg(scene, coarse, tuned):
    """RMS error of surface GHI, direct irradiance and heating rate against a
    2048-photon/column reference, for uniform random (Philox) and scrambled
    Sobol start positions (Sec. 2.3) at 4, 16 and 64 photons/column, with the
    transport time of each; the speed-up is the Philox time needed to reach the
    Sobol error (RMSE ~ a / sqrt(ppc) and time ~ t0 + t1 ppc fitted on the
    Philox runs)."""
    import torch
    from paper_2208_05247_b300 import rt
    stream = torch.cuda.current_stream()
    opts = {k: v for k, v in (tuned or {}).items() if k != "coarse"}

    def run(birth, ppc, seed):
        with rt.Tracer.from_scene(scene, *coarse, stream=stream, birth=birth, **opts) as t:
            t.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.trace(SZA, AZ, F0, ppc * scene.ncol, seed)
            e1.record(stream)
            f = t.fields()
            hr = t.heating_rate()
            return {"ghi": f["sfc_dir"] + f["sfc_dif"], "dir": f["sfc_dir"], "hr": hr}, e0.elapsed_time(e1)

    truth, _ = run(rt.RT_BIRTH_SOBOL, 2048, SEED + 500)
    res = {}
    for name, birth in (("philox", rt.RT_BIRTH_PHILOX), ("sobol", rt.RT_BIRTH_SOBOL)):
        res[name] = {}
        for q, ppc in enumerate((4, 16, 64)):
            run(birth, ppc, SEED + 600)                      # warm
            f, ms = run(birth, ppc, SEED + 601 + q)
            res[name][ppc] = {k: float(np.sqrt(np.mean((f[k] - truth[k]) ** 2))) for k in f}
            res[name][ppc]["ms"] = ms
    ppcs = np.array([4, 16, 64], float)
    t_fit = np.polyfit(ppcs, [res["philox"][p]["ms"] for p in (4, 16, 64)], 1)
    speed = {}
    for k in ("ghi", "dir", "hr"):
        a = np.mean([res["philox"][p][k] * np.sqrt(p) for p in (4, 16, 64)])
        need = (a / res["sobol"][16][k]) ** 2
        speed[k] = float(np.polyval(t_fit, need) / res["sobol"][16]["ms"])
    return {"workload": "benchmark scene, sza 30, reference 2048 photons/column (Sobol, independent scramble)",
            "rmse": res, "speedup_at_16ppc": speed}


# ---- batched spectral + multi-scene workload (one recorded graph per step) ------------------

def batched_leg(steps: int):
    """All 112 quadrature points of 4 scenes of uneven size (128x128x96,
    192x96x128, 256x256x128, 64x64x64) in one persistent launch of 2^26
    photons with energy-proportional budgets, recorded once as a CUDA graph
    (rt_batch_step) and replayed per step; the same step through
    rt_trace_batch for comparison."""
    import torch
    from paper_2208_05247_b300 import rt, scenes
    stream = torch.cuda.current_stream()
    scs = scenes.batch_scenes()
    scale, flux = scenes.gpoint_table()
    tracers = []
    for sc in scs:
        t = rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, stream=stream)
        t.set_options(batch_optics=1)
        t.set_optics(*sc.fields())
        t.set_surface(sc.albedo)
        t.build_accel(2, 2, 2)
        tracers.append(t)
    jobs = [dict(scene=t, sza_deg=SZA, azimuth_deg=AZ, toa_flux=float(flux[g]), gas_scale=float(scale[g]))
            for t in tracers for g in range(len(flux))]
    total = 2 ** 26

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(k):
            fn(i)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    def eager(i):
        for t in tracers:
            t.reset()
        rt.rt_trace_batch(jobs, total_photons=total, seed=SEED + i)

    # a second set of handles on its own stream, with its own recorded step:
    # replays that alternate between the two sets overlap one step's tail
    # with the next step
    s_a, s_b = torch.cuda.Stream(), torch.cuda.Stream()
    tracers_b = []
    for sc in scs:
        t = rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, stream=s_b)
        t.set_options(batch_optics=1)
        t.set_optics(*sc.fields())
        t.set_surface(sc.albedo)
        t.build_accel(2, 2, 2)
        tracers_b.append(t)
    jobs_b = [dict(j, scene=tracers_b[tracers.index(j["scene"])]) for j in jobs]

    def timed_two(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s_a.wait_stream(stream)
        s_b.wait_stream(stream)
        for i in range(k):
            fn(i)
        stream.wait_stream(s_a)
        stream.wait_stream(s_b)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    step = rt.rt_batch_step_create(jobs, total_photons=total)
    step_b = rt.rt_batch_step_create(jobs_b, total_photons=total)
    try:
        for i in range(2):
            rt.rt_batch_step_launch(step, SEED + i)
        ms_graph = timed(lambda i: rt.rt_batch_step_launch(step, SEED + i), steps)
        sts = [t.stats() for t in tracers]
        for t in tracers:
            t.set_stream(s_a)
        two = lambda i: rt.rt_batch_step_launch(step if i % 2 == 0 else step_b, SEED + i)   # noqa: E731
        for i in range(4):
            two(i)
        ms_two = timed_two(two, 2 * ((steps + 1) // 2))
        sts_two = [t.stats() for t in tracers + tracers_b]
        for t in tracers:
            t.set_stream(stream)
    finally:
        rt.rt_batch_step_destroy(step)
        rt.rt_batch_step_destroy(step_b)
    eager(0)
    ms_eager = timed(eager, steps)
    ev = sum(st["events"] for st in sts)
    cr = sum(st["crossings"] for st in sts)
    ph = sum(st["photons"] for st in sts)
    peak, _ = peaks()
    closure = [abs(st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
                   - st["energy_toa_up"] - st["energy_atm_abs"] - st["energy_sfc_abs"]) / st["energy_in"]
               for st in sts + sts_two]
    for t in tracers + tracers_b:
        t.close()
    alg = ev * BYTES_PER_EVENT + cr * BYTES_PER_CROSSING
    return {"workload": "4 scenes (128x128x96, 192x96x128, 256x256x128, 64x64x64) x 112 quadrature points, "
                        "2^26 photons per step, coarse grid 2x2x2, one persistent launch",
            "ms_per_step_graph": ms_graph, "ms_per_step_eager": ms_eager, "photons_per_step": ph,
            "events_per_s": ev / (ms_graph / 1e3), "photons_per_s": ph / (ms_graph / 1e3),
            "roofline_frac": alg / (ms_graph / 1e3) / 1e9 / peak,
            "roofline_note": "algorithmic bytes of the step over the whole replayed step (tally resets included)",
            "two_streams": {"ms_per_step_graph": ms_two, "events_per_s": ev / (ms_two / 1e3),
                            "photons_per_s": ph / (ms_two / 1e3), "roofline_frac": alg / (ms_two / 1e3) / 1e9 / peak,
                            "note": "replays alternate between two sets of the four scene handles and two "
                                    "recorded steps, one stream each (events per step from the one-stream run)"},
            "ledger_residual_max": max(closure), "capped": sum(st["capped"] for st in sts + sts_two)}


# ---- end to end through the C ABI with plain host buffers ------------------------------

def c_abi_host_leg(scene, coarse, tuned, steps, N, begin, total):
    """The step a C caller with ordinary (pageable) host buffers makes: optics
    and albedo in with RT_HOST, grid, reset, trace, and the fields and heating
    rate out with RT_HOST (those calls synchronise), timed on the wall clock."""
    from paper_2208_05247_b300 import rt
    ins = [np.ascontiguousarray(a, dtype=np.float32) for a in scene.fields()]
    alb = np.ascontiguousarray(scene.albedo, dtype=np.float32)
    outs = {"abs3d": np.empty(scene.ncell), "hr": np.empty(scene.ncell)}
    for k in ("sfc_dir", "sfc_dif", "toa_up"):
        outs[k] = np.empty(scene.ncol)
    with rt.Tracer(scene.nx, scene.ny, scene.nz, scene.dx, scene.dy, scene.dz) as t:
        if tuned:
            t.set_options(**{k: v for k, v in tuned.items() if k != "coarse"})

        def one():
            rt.rt_set_optics(t.h, scene.ncell, *ins)
            rt.rt_set_surface(t.h, scene.ncol, alb)
            rt.rt_build_accel(t.h, *coarse)
            rt.rt_reset_tallies(t.h)
            rt.rt_trace_range(t.h, SZA, AZ, F0, begin, N, total, SEED)
            rt.rt_fields(t.h, scene.ncell, scene.ncol, outs["abs3d"], outs["sfc_dir"], outs["sfc_dif"], outs["toa_up"])
            rt.rt_heating_rate(t.h, scene.ncell, outs["hr"], 0)

        one()
        events = t.stats()["events"]
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        dt = (time.perf_counter() - t0) / steps
    h2d = sum(a.nbytes for a in ins) + alb.nbytes
    d2h = sum(v.nbytes for v in outs.values())
    return {"value": events / dt, "unit": UNIT, "ms_per_step": 1e3 * dt, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "buffers": "pageable numpy arrays through RT_HOST, no overlap"}


# ---- our CUDA path --------------------------------------------------------------------

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2208_05247_b300 import build, rt, scenes
    build.build()
    scene = scenes.cumulus_scene(seed=1)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ncell, ncol = scene.ncell, scene.ncol
    d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in scene.fields()]
    d_alb = torch.from_numpy(scene.albedo).to(dev)
    d_out = {"abs3d": torch.empty(ncell, dtype=torch.float64, device=dev),
             "hr": torch.empty(ncell, dtype=torch.float64, device=dev)}
    for k in ("sfc_dir", "sfc_dif", "toa_up"):
        d_out[k] = torch.empty(ncol, dtype=torch.float64, device=dev)
    from paper_2208_05247_b300 import shard
    begin, N, total = shard.photon_range(rank, world, args.ppc * ncol)

    t = rt.Tracer(scene.nx, scene.ny, scene.nz, scene.dx, scene.dy, scene.dz, stream=stream)
    t.set_optics(*d_in)
    t.set_surface(d_alb)
    coarse = tuple(args.coarse) if args.coarse else COARSE
    tuned = None
    if args.launch:
        tuned = {"coarse": list(coarse), "ready_threshold": args.launch[0], "max_inner": args.launch[1],
                 "refill_chunk": args.launch[2], "block_size": 64, "blocks_per_sm": 0}
        t.set_options(**{k: v for k, v in tuned.items() if k != "coarse"})
    elif not args.no_autotune and not args.coarse:
        # untimed: pick coarse factors and launch parameters by photons/s
        from paper_2208_05247_b300 import autotune
        tuned, _ = autotune.autotune(t, args.sza, AZ, F0, N, seed=SEED + 1000)
        coarse = tuned["coarse"]

    def step(seed, ev=None, inputs=None, outputs=None):
        src = inputs if inputs is not None else (d_in, d_alb)
        out = outputs if outputs is not None else d_out
        t.set_optics(*src[0])
        t.set_surface(src[1])
        t.build_accel(*coarse)
        t.reset()
        if ev is not None:
            ev[0].record(stream)
        t.trace_range(args.sza, AZ, F0, begin, N, total, seed)
        if ev is not None:
            ev[1].record(stream)
        rt.rt_fields(t.h, ncell, ncol, out["abs3d"], out["sfc_dir"], out["sfc_dif"], out["toa_up"])
        rt.rt_heating_rate(t.h, ncell, out["hr"], 0)
        if reduce:
            shard.reduce_fields(out)

    reduce = dist is not None and args.reduce_fields
    for _ in range(max(1, args.warmup)):
        step(SEED)
    torch.cuda.synchronize()
    ref_stats = t.stats()
    clocks = Clocks(local)

    def timed(run, k):
        """k steps of `run`, bracketed by a barrier and a device synchronize,
        timed by CUDA events on the default stream (max over ranks)."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        run(k)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        if dist is not None:
            v = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(v, op=dist.ReduceOp.MAX)
            ms = float(v.item())
        return ms

    # (1) one handle on one stream: the steps run one after the other, and the
    # transport launches' CUDA-event durations give the kernel's roofline
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks.start()

    def serial(k):
        for i in range(k):
            step(SEED, evs[i])
    ms_serial = timed(serial, args.steps)
    trace_ms = [a.elapsed_time(b) for a, b in evs]
    st = t.stats()
    assert st["events"] == ref_stats["events"], "event count changed between identical steps"
    assert st["status"] == 0, "transport reported a capped photon"

    # (2) the product path: steps alternate between `streams` handles, one
    # stream each (pipeline.StepRing), so that a step's transport starts on the
    # SMs that the previous step's tail leaves idle
    ring = None
    ms = ms_serial
    if args.streams > 1:
        from paper_2208_05247_b300 import pipeline
        extra = []
        for _ in range(args.streams - 1):
            t2 = rt.Tracer(scene.nx, scene.ny, scene.nz, scene.dx, scene.dy, scene.dz)
            if tuned:
                t2.set_options(**{k: v for k, v in tuned.items() if k != "coarse"})
            extra.append(t2)
        ring = pipeline.StepRing([t] + extra, coarse)
        after = (lambda s, o: shard.reduce_fields(o)) if reduce else None

        def ring_steps(k):
            ring.wait_on(stream)
            for _ in range(k):
                ring.submit(d_in, d_alb, args.sza, AZ, F0, N, SEED, photon_begin=begin, photons_total=total,
                            after=after)
            ring.join(stream)
        ring_steps(max(2, args.warmup) * args.streams)
        torch.cuda.synchronize()
        ms = timed(ring_steps, args.steps)
        for tr in ring.ts:
            s2 = tr.stats()
            assert s2["events"] == ref_stats["events"], "a ring handle traced different histories"
            assert s2["status"] == 0, "transport reported a capped photon"
        t.set_stream(stream)
    clk = clocks.stop()

    events = st["events"]
    crossings = st["crossings"]
    ms_max, events_all = ms, events
    if dist is not None:
        e = torch.tensor([events], dtype=torch.float64, device=dev)
        dist.all_reduce(e)
        events_all = int(e.item())
    value = events_all * args.steps / (ms_max / 1e3)

    # transport kernel roofline (this rank)
    tk = statistics.mean(trace_ms) / 1e3
    alg_bytes = events * BYTES_PER_EVENT + crossings * BYTES_PER_CROSSING
    peak, peak_src = peaks()
    achieved = alg_bytes / tk / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profiled_traffic(), "peak_source": peak_src,
            "kernel": "trace_kernel<double>", "kernel_ms": 1e3 * tk,
            "algorithmic_bytes_per_launch": alg_bytes, "events_per_launch": events, "box_steps_per_launch": crossings,
            # the same launch at sector granularity (a random 16-byte gather, an
            # 8-byte tally update and a 4-byte box word each move a 32-byte sector)
            "sector_bytes_per_launch": events * 64 + crossings * 32,
            "sector_frac": (events * 64 + crossings * 32) / tk / 1e9 / peak,
            "kernel_ms_source": "CUDA events around each transport launch of the single-stream timed loop "
                                "(one launch on the GPU at a time)",
            # the same bytes over the whole product step (all kernels, with the
            # handles' steps overlapping): what the timed `value` reaches
            "step_achieved": alg_bytes / (ms / args.steps / 1e3) / 1e9,
            "step_frac": alg_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
            "photons_per_s": N * world * args.steps / (ms_max / 1e3)}
    # the same algorithmic bytes against this GPU's L2 read bandwidth, measured
    # here (outside the timed region) by the library's read probe: the
    # transport kernel's working set is L2-resident
    l2roof = None
    if not args.no_l2_probe:
        from paper_2208_05247_b300 import mem_probe
        rows = mem_probe.sweep((48, 1024), target_bytes=4 << 30, repeats=3)
        l2roof = {"bound": "l2", "achieved": achieved, "peak": rows[0]["gbs"], "unit": "GB/s",
                  "frac": achieved / rows[0]["gbs"], "dram_read_gbs": rows[1]["gbs"],
                  "peak_source": "rt_probe_read in this run: L2-cached 16-byte reads of a 48 MB buffer "
                                 "(1024 MB for the DRAM figure)"}

    # end to end through the C ABI with host buffers: every step copies its
    # inputs in from pinned host memory and its fields out to pinned host
    # memory; HostPipeline overlaps those copies with the neighbouring steps'
    # transport (two device buffer sets, a copy stream and the tracer's stream)
    e2e = None
    if not args.no_e2e:
        from paper_2208_05247_b300 import pipeline
        h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in scene.fields()]
        h_alb = torch.from_numpy(scene.albedo).pin_memory()
        h_outs = [{k: torch.empty(v.numel(), dtype=torch.float64).pin_memory() for k, v in d_out.items()}
                  for _ in range(2)]
        pipe = pipeline.HostPipeline(ring.ts if ring is not None else t, coarse)
        pipe.submit(h_in, h_alb, args.sza, AZ, F0, N, SEED, h_outs[0], photon_begin=begin, photons_total=total)
        pipe.synchronize()
        assert all(tr.stats()["events"] == events for tr in pipe.ts), "pipelined step traced different histories"
        barrier()
        k2 = max(3, args.steps // 2)
        t0 = time.perf_counter()
        for i in range(k2):
            pipe.submit(h_in, h_alb, args.sza, AZ, F0, N, SEED, h_outs[i & 1], photon_begin=begin,
                        photons_total=total)
        pipe.synchronize()
        dt = time.perf_counter() - t0
        t.set_stream(stream)
        barrier()
        if dist is not None:
            v = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(v, op=dist.ReduceOp.MAX)
            dt = float(v.item())
        h2d = sum(a.numel() * 4 for a in h_in) + h_alb.numel() * 4
        d2h = sum(v.numel() * 8 for v in h_outs[0].values())
        e2e = {"value": events_all * k2 / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / k2,
               "pipelined": "copies of step k+1 in and k-1 out overlap step k's transport (HostPipeline); "
                            f"steps alternate between {len(pipe.ts)} handle(s), one stream each",
               "photons_per_s": N * world * k2 / dt}
        # the same step as a C caller with plain host buffers makes it
        e2e["c_abi_host"] = c_abi_host_leg(scene, coarse, tuned, max(3, args.steps // 4), N, begin, total)

    cstep = births = batched = sweep = None
    if world == 1 and not args.no_sweep:
        sweep = sweep_leg(t, coarse)
    if world == 1 and not args.no_batched:
        batched = batched_leg(max(3, args.steps // 4))
    if world == 1 and not args.no_coupled:
        cstep = coupled_step_leg(t, d_in, d_alb, d_out, N, ms_serial / args.steps, events, max(3, args.steps // 2))
    if world == 1 and not args.no_birth:
        births = birth_leg(scene, coarse, tuned)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        tot, dt, cores = oracle_sample(scene, args.cpu_sample_ppc, SEED + 7)
        cpu = {"value": tot["collisions"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample_ppc} photons/column ({tot['photons']} photons) of the benchmark "
                         f"scene, {dt:.1f} s wall; oracle collisions are all real (analog tracer)",
               "photons_per_s": tot["photons"] / dt}
    dn = None
    if world == 1 and not args.no_denoise:
        dn = denoise_leg(args)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, world, coarse), launch=tuned or "defaults",
                           streams=f"{args.streams} tracer handle(s), one stream each; steps alternate between them",
                           **({"parallelism": f"photon ranges, {world} ranks, fields summed every step "
                                              "(NCCL all-reduce, FP64)"} if reduce else {})),
            "photons_per_s": N * world * args.steps / (ms_max / 1e3),
            "real_scatters_per_s": st["scatters"] * world * args.steps / (ms_max / 1e3),
            "events_per_step": events_all, "real_scatter_fraction": st["scatters"] / max(1, events),
            "trace_kernel_ms": 1e3 * tk, "serial_ms_per_step": ms_serial / args.steps,
            "serial_events_per_s": events_all * args.steps / (ms_serial / 1e3), "clocks": clk, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": KERNELS_PER_STEP * args.steps, "sobol_birth": births, "coupled_step": cstep,
            "l2_roofline": l2roof, "time_to_rmse": dn, "batched": batched, "config1_sweep": sweep}
    print(json.dumps(line), flush=True)
    for tr in (ring.ts if ring is not None else [t]):
        tr.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
