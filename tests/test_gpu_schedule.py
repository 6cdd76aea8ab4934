"""GPU tests of the launch order (rt_options.schedule): starting the photons of
the optically thickest columns first changes when each photon runs, never what
it does, because a photon's history depends only on its id."""
import numpy as np
import pytest

from paper_2208_05247_b300 import rt, scenes

pytestmark = pytest.mark.gpu

FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")
COUNTERS = ("photons", "events", "scatters", "crossings", "surface_hits", "roulette_kills", "max_events_photon")


def run(scene, schedule, ranges, total, birth=rt.RT_BIRTH_PHILOX):
    with rt.Tracer.from_scene(scene, 4, 4, 4, schedule=schedule, birth=birth) as t:
        t.build_accel(4, 4, 4)          # the schedule applies from the next grid build
        t.reset()
        for b, c in ranges:
            t.trace_range(35.0, 120.0, 1000.0, b, c, total, 17)
        return t.fields(split=True), t.stats()


@pytest.mark.parametrize("birth", [rt.RT_BIRTH_PHILOX, rt.RT_BIRTH_SOBOL])
def test_thick_first_changes_no_history(small_scene, birth):
    sc = small_scene
    total = 128 * sc.ncol
    # whole rounds of >= 64 photons per column (ordered launches), rounds below
    # that (id order), and an unaligned split (id order)
    half = 64 * sc.ncol
    for ranges in ([(0, total)], [(0, half), (half, total - half)], [(0, 8 * sc.ncol), (8 * sc.ncol, total - 8 * sc.ncol)],
                   [(0, 5000), (5000, total - 5000)]):
        f0, s0 = run(sc, rt.RT_SCHEDULE_IDS, ranges, total, birth)
        f1, s1 = run(sc, rt.RT_SCHEDULE_THICK_FIRST, ranges, total, birth)
        for k in COUNTERS:
            assert s0[k] == s1[k], (ranges, k)
        for k in FIELDS:
            scale = np.abs(f0[k]).max()
            assert np.allclose(f1[k], f0[k], rtol=1e-12, atol=1e-12 * scale), (ranges, k)


def test_thick_first_on_a_ragged_coarse_grid():
    """nx, ny not multiples of the coarse factors: the last coarse columns are narrower."""
    sc = scenes.cumulus_scene(seed=3, nx=37, ny=23, nz=16)
    total = 64 * sc.ncol
    out = []
    for sched in (rt.RT_SCHEDULE_IDS, rt.RT_SCHEDULE_THICK_FIRST):
        with rt.Tracer.from_scene(sc, 4, 4, 4, schedule=sched) as t:
            t.build_accel(8, 8, 4)
            t.reset()
            t.trace(20.0, 0.0, 1000.0, total, 3)
            out.append((t.fields(), t.stats()))
    assert out[0][1]["events"] == out[1][1]["events"] and out[0][1]["photons"] == total
    for k in ("abs3d", "sfc_dir", "sfc_dif", "toa_up"):
        assert np.allclose(out[1][0][k], out[0][0][k], rtol=1e-12, atol=1e-12 * np.abs(out[0][0][k]).max())
