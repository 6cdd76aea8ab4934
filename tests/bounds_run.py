"""Runs the tracer's launch paths against the bounds-checking build of the
library (RT_CHECK_BOUNDS=1, path in the environment variable RT_LIB) and
prints one JSON line: the status of every case. Every gather, tally and box
index of the transport kernel is checked there, and a failed check sets
RT_E_BOUNDS instead of trapping. Used by tests/test_gpu_bounds.py in a
subprocess, so that this process loads only the checking library."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2208_05247_b300 import rt, scenes  # noqa: E402

rt.LIB = os.environ["RT_LIB"]
results = {}


def record(name, fn):
    try:
        results[name] = fn()
    except rt.RtError as e:
        results[name] = e.code


def handle_case(sc, coarse, photons, begin=0, total=None, diffuse=0.0, sza=30.0, az=20.0, **opts):
    def run():
        with rt.Tracer.from_scene(sc, *coarse, **opts) as t:
            if diffuse:
                rt.rt_trace_ex(t.h, sza, az, 1000.0, diffuse, begin, photons, total or begin + photons, 3)
            else:
                t.trace_range(sza, az, 1000.0, begin, photons, total or begin + photons, 3)
            t.fields(split=True)
            t.heating_rate()
            st = t.stats()
            return st["status"] if st["photons"] == photons else -100
    return run


small = scenes.ellipsoid_scene(seed=0)
ragged = scenes.cumulus_scene(seed=5, nx=48, ny=40, nz=30)
for coarse in ((0, 0, 0), (1, 1, 1), (5, 3, 7), (32, 32, 32)):
    record("ellipsoid_coarse_%d_%d_%d" % coarse, handle_case(small, coarse, 2 ** 18))
for coarse in ((2, 2, 2), (5, 3, 7), (48, 40, 30)):
    record("ragged_coarse_%d_%d_%d" % coarse, handle_case(ragged, coarse, 64 * ragged.ncol))
record("ellipsoid_ids_beyond_2_32", handle_case(small, (0, 0, 0), 192 * small.ncol,
                                                begin=(1 << 32) - 96 * small.ncol))
record("ellipsoid_sobol", handle_case(small, (0, 0, 0), 2 ** 18, birth=rt.RT_BIRTH_SOBOL))
record("ellipsoid_fp32_tallies", handle_case(small, (0, 0, 0), 2 ** 18, tally_precision=rt.RT_TALLY_FP32))
record("ellipsoid_literal_scatterer", handle_case(small, (0, 0, 0), 2 ** 18, pcld_mode=rt.RT_PCLD_EXTINCTION))
record("ellipsoid_diffuse_top", handle_case(small, (0, 0, 0), 2 ** 18, diffuse=0.4))
record("ellipsoid_sun_overhead", handle_case(small, (0, 0, 0), 2 ** 18, sza=0.0, az=0.0))
record("ellipsoid_aggregated_flush", handle_case(small, (0, 0, 0), 2 ** 18, tally_aggregate=1))


def batched():
    ts = []
    for sc in (small, ragged):
        t = rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz)
        t.set_options(batch_optics=1)
        t.set_optics(*sc.fields())
        t.set_surface(sc.albedo)
        t.build_accel(2, 2, 2)
        ts.append(t)
    jobs = [dict(scene=t, sza_deg=30.0 + 10 * j, azimuth_deg=40.0 * j, toa_flux=200.0 + 50 * j, gas_scale=g)
            for t in ts for j, g in enumerate((0.001, 0.5, 8.0))]
    rt.rt_trace_batch(jobs, total_photons=2 ** 20, seed=4)
    out = [t.stats()["status"] for t in ts]
    for t in ts:
        t.close()
    return min(out) if min(out) < 0 else max(out)


def step():
    sc = ragged
    dev = torch.device("cuda")
    with rt.Tracer.from_scene(sc, 5, 3, 7) as t:
        inp = [torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev) for a in sc.fields()]
        alb = torch.from_numpy(sc.albedo.ravel()).to(dev)
        out = {k: torch.zeros(sc.ncell if k in ("abs3d", "hr") else sc.ncol, dtype=torch.float64, device=dev)
               for k in ("abs3d", "hr", "sfc_dir", "sfc_dif", "toa_up")}
        s = rt.rt_step_create(t.h, sc.ncell, sc.ncol, inp, 64 * sc.ncol, albedo=alb, **out)
        try:
            for k in range(2):
                rt.rt_step_launch(s, 40.0, 10.0, 1000.0, 0.2, 7 + k)
                rt.rt_synchronize(t.h)
        finally:
            rt.rt_step_destroy(s)
        return t.stats()["status"]


def noalloc():
    sc = ragged
    dev = torch.device("cuda")
    f = [torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev) for a in sc.fields()]
    alb = torch.from_numpy(sc.albedo.ravel()).to(dev)
    o = [torch.zeros(sc.ncell, dtype=torch.float64, device=dev) for _ in range(2)] + \
        [torch.zeros(sc.ncol, dtype=torch.float64, device=dev) for _ in range(3)]
    rt.rt_trace_noalloc(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, *f, alb, 35.0, 60.0, 1000.0, 64 * sc.ncol, 9,
                        *o, coarse=(5, 3, 7))
    return 0


record("batched_two_scenes", batched)
record("coupled_step", step)
record("noalloc", noalloc)
big = scenes.cumulus_scene(seed=1)
record("cumulus_256_4ppc", handle_case(big, (2, 2, 2), 4 * big.ncol))
record("cumulus_256_64ppc_thick_first", handle_case(big, (2, 2, 2), 64 * big.ncol, ready_threshold=16, block_size=64,
                                                    max_inner=64, refill_chunk=128))
print(json.dumps(results), flush=True)
