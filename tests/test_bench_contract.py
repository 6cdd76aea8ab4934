"""Host-side contracts, without a GPU: the bench's reference arm (the CPU
oracle timed on a bounded sample) prints the benchmark's JSON line, and the
launch autotuner only leaves its starting configuration for a clear gain."""
import json
import os
import subprocess
import sys

import pytest

from paper_2208_05247_b300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "photons_per_s"):
        assert k in d, k
    assert d["value"] > 0 and d["photons_per_s"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "events/s" and d["higher_is_better"] is True and d["vs_baseline"] is None
    # the bounded sample is stated, and traced photons are counted as such
    assert "1 photon/column" in d["config"]["sample"]
    assert d["config"]["photons_per_step_traced"] == 256 * 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


class _FakeTracer:
    nx, ny, nz = 256, 256, 128

    def __init__(self):
        self.options, self.coarse = None, None

    def set_options(self, **kw):
        self.options = kw

    def build_accel(self, cx, cy, cz):
        self.coarse = (cx, cy, cz)


@pytest.mark.parametrize("gain, moves", [(0.01, False), (0.05, True)])
def test_autotune_needs_a_clear_gain_to_move(monkeypatch, gain, moves):
    """One candidate (box_levels 3) is faster than the start by `gain`, every
    other one slower: below the 2 % hysteresis the start is kept."""
    def fake_time(tracer, sza, az, flux, photons, seed, coarse, repeats=2, **opts):
        ms = 10.0
        if opts.get("box_levels") == 3 and tuple(coarse) == (2, 2, 2):
            ms = 10.0 / (1.0 + gain)
        elif (tuple(coarse) != (2, 2, 2) or opts.get("box_levels") != 4 or opts.get("ready_threshold") != 16
              or opts.get("max_inner") != 64 or opts.get("refill_min") != 8 or opts.get("refill_chunk") != 128
              or opts.get("block_size") != 64 or opts.get("blocks_per_sm") != 0):
            ms = 12.0
        return ms, {"events": 1000, "crossings": 3000}
    monkeypatch.setattr(autotune, "time_config", fake_time)
    t = _FakeTracer()
    best, table = autotune.autotune(t, 30.0, 0.0, 1000.0, 1 << 20)
    assert best["box_levels"] == (3 if moves else 4)
    assert t.coarse == (2, 2, 2) and t.options["box_levels"] == best["box_levels"]
    assert len(table) > 10
