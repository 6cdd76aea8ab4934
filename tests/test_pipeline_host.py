"""Host-side checks of the overlapped-step helpers (no GPU): the handle list
is validated before any stream or buffer is made."""
from types import SimpleNamespace

import pytest

from paper_2208_05247_b300 import pipeline


def _fake(nz):
    return SimpleNamespace(nx=8, ny=8, nz=nz, ncell=64 * nz, ncol=64)


@pytest.mark.parametrize("cls", [pipeline.StepRing, pipeline.HostPipeline])
def test_handles_must_share_the_grid(cls):
    with pytest.raises(ValueError, match="same grid"):
        cls([_fake(4), _fake(5)])


@pytest.mark.parametrize("cls", [pipeline.StepRing, pipeline.HostPipeline])
def test_no_handles_is_an_error(cls):
    with pytest.raises(ValueError, match="no tracer"):
        cls([])
