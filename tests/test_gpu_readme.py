"""The Python usage examples in README.md run as written on the GPU."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _python_blocks():
    text = open(os.path.join(ROOT, "README.md")).read()
    return re.findall(r"```python\n(.*?)```", text, flags=re.S)


def test_readme_has_python_examples():
    assert len(_python_blocks()) >= 2


@pytest.mark.parametrize("k", range(2))
def test_readme_python_example_runs(k):
    ns = {}
    exec(compile(_python_blocks()[k], "README.md example %d" % k, "exec"), ns)
    if "fields" in ns and isinstance(ns["fields"], dict):        # the single-trace example
        assert ns["fields"]["sfc_dir"].mean() > 0.0 and ns["hr"].shape == ns["fields"]["abs3d"].shape
    if "ring" in ns:                                             # the two-handle step loop
        ns["ring"].synchronize()
        assert [t.stats()["status"] for t in ns["ring"].ts] == [0, 0]
        assert float(ns["out"]["sfc_dir"].mean()) > 0.0
