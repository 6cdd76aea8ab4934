"""Precision study on the LES-like cumulus scene (256x256x128) at 64 photons
per column, sza 30: FP32 transport with FP64 tallies (the default), FP32
transport with FP32 tallies, and the FP64 CPU oracle. Errors are stated per
output field: the deterministic FP32-vs-FP64 tally difference (same photon
histories) and the difference of each GPU variant from the oracle (bias with
its standard error, and RMS against the RMS the sampling noise alone predicts).
The table is printed (run pytest with -s to see it).
"""
import json

import numpy as np
import pytest

import oracle
from paper_2208_05247_b300 import rt, scenes

pytestmark = pytest.mark.gpu

FIELDS = ("hr", "sfc_dir", "sfc_dif", "toa_up")


def _gpu(scene, precision, seeds, N):
    out = {f: [] for f in FIELDS}
    closure = []
    with rt.Tracer.from_scene(scene, 4, 4, 8, tally_precision=precision) as t:
        for s in seeds:
            t.reset()
            t.trace(30.0, 0.0, 1000.0, N, s)
            f = t.fields()
            out["hr"].append(t.heating_rate(0))
            for k in ("sfc_dir", "sfc_dif", "toa_up"):
                out[k].append(f[k])
            st = t.stats()
            lhs = st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
            rhs = st["energy_toa_up"] + st["energy_atm_abs"] + st["energy_sfc_abs"]
            closure.append((lhs - rhs) / st["energy_in"])
    return {k: np.stack(v) for k, v in out.items()}, np.array(closure)


def _oracle(scene, seeds, N):
    out = {f: [] for f in FIELDS}
    for s in seeds:
        r = oracle.trace(scene, 30.0, 0.0, 1000.0, N, s)
        out["hr"].append(oracle.heating_rate(r.abs3d, scene.dz))
        for k in ("sfc_dir", "sfc_dif", "toa_up"):
            out[k].append(getattr(r, k))
    return {k: np.stack(v) for k, v in out.items()}


def _vs(a, b):
    """bias, its SE, RMS difference of the means, and the RMS noise alone predicts."""
    ma, mb = a.mean(0), b.mean(0)
    va = a.var(0, ddof=1) / a.shape[0]
    vb = b.var(0, ddof=1) / b.shape[0]
    d = ma - mb
    bias = float(d.mean())
    bias_se = float(np.sqrt((a.reshape(a.shape[0], -1).mean(1).var(ddof=1) / a.shape[0]) +
                            (b.reshape(b.shape[0], -1).mean(1).var(ddof=1) / b.shape[0])))
    return {"bias": bias, "bias_se": bias_se, "rms": float(np.sqrt((d ** 2).mean())),
            "rms_noise": float(np.sqrt((va + vb).mean())), "mean_ref": float(mb.mean())}


def test_precision_study_cumulus():
    sc = scenes.cumulus_scene(seed=1)
    N = 64 * sc.ncol
    seeds = list(range(40, 48))
    g64, c64 = _gpu(sc, rt.RT_TALLY_FP64, seeds, N)
    g32, c32 = _gpu(sc, rt.RT_TALLY_FP32, seeds, N)
    orc = _oracle(sc, range(900, 904), N)
    table = {"workload": "cumulus 256x256x128, sza 30, 64 photons/column", "fields": {}}
    for f in FIELDS:
        d = g32[f] - g64[f]
        scale = np.abs(g64[f]).max()
        row = {"fp32_vs_fp64_tally": {"max_abs": float(np.abs(d).max()), "max_rel_to_field_max": float(np.abs(d).max() / scale),
                                      "rms": float(np.sqrt((d ** 2).mean()))},
               "fp64_tally_vs_oracle": _vs(g64[f], orc[f]),
               "fp32_tally_vs_oracle": _vs(g32[f], orc[f])}
        table["fields"][f] = row
        # the tally precision moves results far less than the sampling noise
        assert row["fp32_vs_fp64_tally"]["rms"] < 0.05 * row["fp64_tally_vs_oracle"]["rms_noise"], (f, row)
        # no bias of the default configuration against the oracle
        r = row["fp64_tally_vs_oracle"]
        assert abs(r["bias"]) < 4 * r["bias_se"] + 1e-12, (f, r)
        # differences are what the noise predicts (no structured error)
        assert r["rms"] < 1.3 * r["rms_noise"], (f, r)
    table["closure_residual"] = {"fp64_tally_max": float(np.abs(c64).max()), "fp32_tally_max": float(np.abs(c32).max())}
    assert np.abs(c64).max() < 1e-9
    print(json.dumps(table, indent=1))
