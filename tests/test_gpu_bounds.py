"""Bounds checking in place of a sanitizer: the tracer's launch paths run
against the library's bounds-checking build (every gather, tally and box
index of the transport kernel checked; a failed check sets RT_E_BOUNDS and
redirects the access in bounds, nothing traps). No case may report it."""
import json
import os
import subprocess
import sys

import pytest

from paper_2208_05247_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_index_leaves_its_array():
    lib = build.build_checked()
    env = dict(os.environ, RT_LIB=lib)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_run.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    res = json.loads([ln for ln in p.stdout.splitlines() if ln.startswith("{")][-1])
    assert len(res) == 19, res
    bad = {k: v for k, v in res.items() if v != 0}
    assert not bad, bad
