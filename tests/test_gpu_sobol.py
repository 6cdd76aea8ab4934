"""GPU tests of the scrambled-Sobol start positions (Sec. 2.3: photons enter the
domain top at the points of a scrambled Sobol sequence).

The Sobol points themselves are integer work, so the device's points must equal
the oracle's bit for bit. The transport with Sobol starts is checked against
the oracle's Sobol-start tracer statistically (independent scrambles per seed
make the batches independent randomised quasi-Monte Carlo replicates), and its
direct-beam error against the oracle's deterministic Beer-Lambert reference.
"""
import numpy as np
import pytest

import oracle
from paper_2208_05247_b300 import rt
from tests import refs

pytestmark = pytest.mark.gpu

FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")


def test_device_sobol_points_equal_the_oracle():
    for k0, n in ((0, 1 << 16), ((1 << 31) - 100, 4096), ((1 << 32) - 64, 64)):
        want = oracle.sobol2(n, k0)
        assert np.array_equal(rt.rt_debug_sobol(k0, n), want)
        sx, sy = 0x9E3779B9, 0x7F4A7C15
        assert np.array_equal(rt.rt_debug_sobol(k0, n, sx, sy), want ^ np.array([sx, sy], dtype=np.uint32))


def gpu_runs(scene, sza, az, photons, seeds, birth):
    out = {k: [] for k in FIELDS}
    with rt.Tracer.from_scene(scene, birth=birth) as t:
        for s in seeds:
            t.reset()
            t.trace(sza, az, 1000.0, photons, s)
            f = t.fields(split=True)
            for k in FIELDS:
                out[k].append(f[k])
    return {k: np.stack(v) for k, v in out.items()}


def test_sobol_transport_parity_with_oracle(small_scene):
    sc = small_scene
    B, N = 8, 64 * sc.ncol
    g = gpu_runs(sc, 40.0, 60.0, N, range(30, 30 + B), rt.RT_BIRTH_SOBOL)
    o = {k: [] for k in FIELDS}
    for s in range(B):
        r = oracle.trace(sc, 40.0, 60.0, 1000.0, N, 500 + s, birth="sobol")
        for k in FIELDS:
            o[k].append(getattr(r, k))
    for k in FIELDS:
        rel, se = refs.domain_compare(g[k], np.stack(o[k]))
        assert abs(rel) < 4 * se + 1e-12, (k, rel, se)


def test_sobol_birth_lowers_the_direct_beam_error(small_scene):
    sc = small_scene
    sza, az = 30.0, 30.0
    truth = 1000.0 * np.cos(np.deg2rad(sza)) * oracle.direct_beam(sc, sza, az, nsub=16)
    N = 16 * sc.ncol
    err = {}
    for birth in (rt.RT_BIRTH_PHILOX, rt.RT_BIRTH_SOBOL):
        r = gpu_runs(sc, sza, az, N, range(70, 86), birth)["sfc_dir"]
        se = r.std(axis=0, ddof=1).mean() / np.sqrt(r.shape[0])
        assert abs(r.mean() - truth.mean()) < 4 * se + 1e-9, birth      # unbiased
        err[birth] = np.sqrt(((r - truth) ** 2).mean())
    assert err[rt.RT_BIRTH_SOBOL] < 0.7 * err[rt.RT_BIRTH_PHILOX], err


def test_sobol_ranges_add_up_to_the_full_run(small_scene):
    """The Sobol index of a photon is its global id div the column count, so
    disjoint id ranges (separate calls or GPUs) reproduce the single run."""
    sc = small_scene
    N = 16 * sc.ncol
    with rt.Tracer.from_scene(sc, birth=rt.RT_BIRTH_SOBOL) as t:
        t.trace(30.0, 0.0, 1000.0, N, 9)
        whole = t.fields(split=True)
        ev = t.stats()["events"]
        t.reset()
        for b, c in ((0, 5000), (5000, N - 5000)):
            t.trace_range(30.0, 0.0, 1000.0, b, c, N, 9)
        parts = t.fields(split=True)
        assert t.stats()["events"] == ev
    for k in FIELDS:
        assert np.allclose(parts[k], whole[k], rtol=1e-12, atol=1e-12 * np.abs(whole[k]).max())
