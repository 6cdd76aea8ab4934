"""Checkpoint files without a GPU: the scene hash sees every input, a
checkpoint round-trips, and resume refuses another scene or run before it
traces anything."""
import copy

import numpy as np
import pytest

from paper_2208_05247_b300 import checkpoint, scenes


def _fake_fields(sc, rng):
    s3, s2 = (sc.nz, sc.ny, sc.nx), (sc.ny, sc.nx)
    return {k: rng.random(s3 if k.startswith("abs") else s2) for k in checkpoint.FIELDS}


def test_scene_hash_sees_every_input():
    sc = scenes.ellipsoid_scene(seed=0)
    h = checkpoint.scene_hash(sc)
    assert h == checkpoint.scene_hash(copy.deepcopy(sc))
    for name in ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld", "albedo"):
        other = copy.deepcopy(sc)
        a = getattr(other, name)
        a.flat[a.size // 2] = np.float32(a.flat[a.size // 2] + 0.01)
        assert checkpoint.scene_hash(other) != h, name
    other = copy.deepcopy(sc)
    other.dz = sc.dz * 1.5
    assert checkpoint.scene_hash(other) != h


def test_checkpoint_round_trip_and_refusals(tmp_path):
    sc = scenes.ellipsoid_scene(seed=0)
    rng = np.random.default_rng(1)
    run = checkpoint.run_params(30.0, 10.0, 1000.0, 1 << 20, 77)
    f = _fake_fields(sc, rng)
    led = {k: (123 if i < 7 else 4.5) for i, k in enumerate(checkpoint.LEDGER)}
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, sc, run, 1 << 19, f, led)
    meta, f2, led2 = checkpoint.load(path)
    assert meta["done"] == 1 << 19 and meta["run"] == run
    assert all(np.array_equal(f[k], f2[k]) for k in checkpoint.FIELDS) and led2 == led

    class NoTrace:
        def __getattr__(self, name):
            raise AssertionError("resume traced before checking the checkpoint")
    other = copy.deepcopy(sc)
    other.k_cld[0, 0, 0] += np.float32(1.0)
    with pytest.raises(ValueError, match="another scene"):
        checkpoint.resume(path, NoTrace(), other, run)
    with pytest.raises(ValueError, match="another run"):
        checkpoint.resume(path, NoTrace(), sc, dict(run, seed=78))
