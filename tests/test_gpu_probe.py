"""The memory-system probe that measures the L2 ceiling of the transport
kernel's roofline: it reads what it is given and separates L2 from DRAM."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2208_05247_b300 import build, mem_probe, rt  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_probe_separates_l2_from_dram_and_checks_arguments():
    rows = mem_probe.sweep((8, 512), target_bytes=2 << 30, repeats=2)
    for r in rows:
        assert math.isfinite(r["gbs"]) and r["gbs"] > 0
    # an 8 MB buffer stays in L2; 512 MB streams from DRAM
    assert rows[0]["gbs"] > 1.2 * rows[1]["gbs"], rows
    buf = torch.zeros(1024, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    for nbytes, reps in ((0, 1), (24, 1), (4096, 0)):
        with pytest.raises(rt.RtError):
            rt.rt_probe_read(buf, nbytes, reps, sink)
