"""Checkpoint and resume of a long trace.

A run of `photons_total` photons is the sum of its parts: the random stream of
a photon depends only on its id and the seed (counter-based Philox), and
rt_trace_range normalises every part by the whole run's photon count, so the
fields of ids [0, done) plus those of [done, total) are the fields of the whole
run up to the order of FP64 additions. A checkpoint therefore holds the fields
and energy ledger of the ids done so far, the run's parameters and a hash of
the scene; `resume` checks both against the caller's and traces the rest.
"""
from __future__ import annotations

import hashlib
import json

import numpy as np

FIELDS = ("abs3d", "abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "sfc_abs", "toa_up")
LEDGER = ("photons", "events", "scatters", "crossings", "surface_hits", "roulette_kills", "capped",
          "energy_in", "energy_toa_up", "energy_atm_abs", "energy_sfc_abs", "energy_created",
          "energy_destroyed", "energy_capped")        # all additive over photon ranges


def scene_hash(scene) -> str:
    """sha256 over the grid, the spacing, the five optics fields and the albedo."""
    h = hashlib.sha256()
    h.update(np.array([scene.nx, scene.ny, scene.nz], dtype=np.int64).tobytes())
    h.update(np.array([scene.dx, scene.dy, scene.dz], dtype=np.float64).tobytes())
    for a in (*scene.fields(), scene.albedo):
        h.update(np.ascontiguousarray(a, dtype=np.float32).tobytes())
    return h.hexdigest()


def run_params(sza_deg, azimuth_deg, toa_flux, photons_total, seed) -> dict:
    return {"sza_deg": float(sza_deg), "azimuth_deg": float(azimuth_deg), "toa_flux": float(toa_flux),
            "photons_total": int(photons_total), "seed": int(seed)}


def trace_part(tracer, run, begin, count):
    """Fields and ledger of photon ids [begin, begin + count) of `run` (the
    tracer's tallies are reset first)."""
    tracer.reset()
    if count:
        tracer.trace_range(run["sza_deg"], run["azimuth_deg"], run["toa_flux"], begin, count, run["photons_total"],
                           run["seed"])
    f = tracer.fields(split=True)
    st = tracer.stats()
    if st["status"] != 0:
        raise RuntimeError("trace part [%d, %d) ended with status %d" % (begin, begin + count, st["status"]))
    return f, {k: st[k] for k in LEDGER}


def save(path, scene, run, done, fields, ledger):
    """Write a checkpoint of ids [0, done) of `run` (fields and ledger summed over them)."""
    meta = {"scene_sha256": scene_hash(scene), "run": run, "done": int(done)}
    np.savez(path, meta=json.dumps(meta), ledger=json.dumps(ledger), **{k: fields[k] for k in FIELDS})


def load(path):
    z = np.load(path, allow_pickle=False)
    meta = json.loads(str(z["meta"]))
    ledger = json.loads(str(z["ledger"]))
    return meta, {k: z[k] for k in FIELDS}, ledger


def combine(a_fields, a_ledger, b_fields, b_ledger):
    f = {k: a_fields[k] + b_fields[k] for k in FIELDS}
    led = {k: a_ledger[k] + b_ledger[k] for k in LEDGER}
    return f, led


def resume(path, tracer, scene, run, chunk=None):
    """Finish the run a checkpoint started: the scene and parameters must be the
    checkpoint's; traces ids [done, photons_total) in chunks of `chunk` (all at
    once by default) and returns (fields, ledger) of the whole run."""
    meta, fields, ledger = load(path)
    if meta["scene_sha256"] != scene_hash(scene):
        raise ValueError("checkpoint belongs to another scene")
    if meta["run"] != run:
        raise ValueError("checkpoint belongs to another run: %r" % (meta["run"],))
    done, total = meta["done"], run["photons_total"]
    step = chunk or (total - done)
    while done < total:
        n = min(step, total - done)
        f, led = trace_part(tracer, run, done, n)
        fields, ledger = combine(fields, ledger, f, led)
        done += n
    return fields, ledger
