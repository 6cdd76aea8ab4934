"""Checkpoint and resume on the GPU: a run traced in part, written to a
checkpoint, and finished by another handle in two chunks equals the run traced
at once (counters exactly, fields and energies to FP64 addition order)."""
import numpy as np
import pytest

from paper_2208_05247_b300 import checkpoint, rt, scenes

pytestmark = pytest.mark.gpu


def test_resumed_run_equals_uninterrupted_run(tmp_path):
    sc = scenes.ellipsoid_scene(seed=0)
    total = 300 * sc.ncol + 17                  # not whole rounds: id order throughout
    run = checkpoint.run_params(35.0, 25.0, 1000.0, total, 2024)
    with rt.Tracer.from_scene(sc) as t:
        f_all, led_all = checkpoint.trace_part(t, run, 0, total)
    done = 123_457
    path = str(tmp_path / "run.npz")
    with rt.Tracer.from_scene(sc) as t:
        f, led = checkpoint.trace_part(t, run, 0, done)
        checkpoint.save(path, sc, run, done, f, led)
    with rt.Tracer.from_scene(sc) as t:               # a fresh handle, as after a restart
        f_res, led_res = checkpoint.resume(path, t, sc, run, chunk=(total - done) // 2 + 1)
    for k in ("photons", "events", "scatters", "crossings", "surface_hits", "roulette_kills", "capped"):
        assert led_res[k] == led_all[k], k
    for k in checkpoint.LEDGER[7:]:
        assert np.isclose(led_res[k], led_all[k], rtol=1e-12, atol=1e-12 * led_all["energy_in"]), k
    for k in checkpoint.FIELDS:
        assert np.allclose(f_res[k], f_all[k], rtol=1e-12, atol=1e-12 * np.abs(f_all[k]).max()), k
