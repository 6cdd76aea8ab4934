"""The largest grid the library takes: 2047 x 2048 x 512 cells (2^31 minus
1.05 M), traced first with the bounds-checking build (no index may leave its
array), then with the normal build, whose domain means must match the same
layers on a 16 x 16 grid (the scene is horizontally homogeneous). ~150 GB of
device memory, built on the device."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2208_05247_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib):
    env = dict(os.environ, RT_LIB=lib)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "maxsize_run.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads([ln for ln in p.stdout.splitlines() if ln.startswith("{")][-1])


def test_largest_grid():
    checked = _run(build.build_checked())
    assert checked["ncell_max"] < checked["limit"] and checked["limit"] - checked["ncell_max"] < 148 * 32 * 256
    for part in ("big", "big_finest", "small"):
        assert all(b["status"] == 0 for b in checked[part]), (part, checked[part])
    res = _run(build.build())
    for part in ("big", "big_finest", "small"):
        for b in res[part]:
            assert b["status"] == 0, (part, b)
            assert b["photons"] == (16 * 16 * 16384 if part == "small" else 2047 * 2048), (part, b)
            assert b["ledger"] < 1e-9, (part, b)
    for k in ("sfc_dir", "sfc_dif", "toa_up", "atm_abs"):
        a = np.array([b[k] for b in res["big"]])
        s = np.array([b[k] for b in res["small"]])
        se = np.sqrt(a.var(ddof=1) / a.size + s.var(ddof=1) / s.size)
        assert abs(a.mean() - s.mean()) < 4.5 * se + 1e-12 * abs(s.mean()), (k, a.mean(), s.mean(), se)
        # the finest coarse grid (one cell per coarse cell) traces the same expectation
        f = res["big_finest"][0][k]
        assert abs(f - s.mean()) < 4.5 * np.sqrt(a.var(ddof=1) + s.var(ddof=1) / s.size) + 1e-12, (k, f, s.mean())
