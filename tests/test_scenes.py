"""The seeded input generators against the recipe they state (CPU only):
grids, the gas profile, cloud optics, cloud cover, the in-cloud extinction
distribution, cloud heights, surface albedo and the g-point table."""
import math

import numpy as np
import pytest

from paper_2208_05247_b300 import scenes


def _layout_ok(sc):
    for a in (*sc.fields(), sc.albedo):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    assert all(a.shape == (sc.nz, sc.ny, sc.nx) for a in sc.fields())
    assert sc.albedo.shape == (sc.ny, sc.nx)


def _cloud_heights(sc):
    zc = (np.arange(sc.nz) + 0.5) * sc.dz
    k = np.nonzero((sc.k_cld > 0).any(axis=(1, 2)))[0]
    return zc[k.min()], zc[k.max()]


def test_gas_profile_values_written_out():
    # 2e-5 exp(-z/8000) at the centres of layers 0 and 31 of 100 m
    k = scenes.gas_profile(32, 100.0)
    assert k[0] == pytest.approx(2e-5 * math.exp(-50.0 / 8000.0), rel=1e-6)
    assert k[31] == pytest.approx(2e-5 * math.exp(-3150.0 / 8000.0), rel=1e-6)
    assert scenes.gas_profile(4, 25.0, scale=3.0)[2] == pytest.approx(3 * 2e-5 * math.exp(-62.5 / 8000.0), rel=1e-6)


def test_ellipsoid_scene_recipe():
    sc = scenes.ellipsoid_scene(seed=0)
    _layout_ok(sc)
    assert (sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz) == (32, 32, 32, 100.0, 100.0, 100.0)
    cloudy = sc.k_cld > 0
    assert 0 < cloudy.sum() < cloudy.size // 4
    assert np.all(sc.k_cld[cloudy] == np.float32(0.05))
    assert np.all(sc.ssa_cld[cloudy] == np.float32(0.999999)) and np.all(sc.g_cld[cloudy] == np.float32(0.86))
    assert not sc.ssa_cld[~cloudy].any() and not sc.g_cld[~cloudy].any()
    assert np.all(sc.ssa_gas == np.float32(0.9)) and np.all(sc.albedo == np.float32(0.2))
    assert np.allclose(sc.k_gas[:, 3, 7], scenes.gas_profile(32, 100.0))
    # radii U(200, 500) m and bases at 800 m: cloud between 800 and 1800 m
    for rx, ry, rz, cx, cy, cz in sc.meta["blobs"]:
        assert 200.0 <= min(rx, ry, rz) and max(rx, ry, rz) <= 500.0
        assert cz - rz == pytest.approx(800.0)
    lo, hi = _cloud_heights(sc)
    assert lo >= 800.0 and hi <= 1800.0


@pytest.mark.parametrize("shape", [(256, 256, 128), (128, 128, 128)])
def test_cumulus_scene_recipe(shape):
    nx, ny, nz = shape
    sc = scenes.cumulus_scene(seed=1, nx=nx, ny=ny, nz=nz)
    _layout_ok(sc)
    assert (sc.dx, sc.dy, sc.dz) == (50.0, 50.0, 25.0)
    # 400 blobs on 256^2 columns, scaled with the area
    assert sc.meta["nblobs"] == round(400 * nx * ny / 256 ** 2)
    # projected cloud cover 20 % (a quantile threshold: exact up to ties)
    assert abs(sc.cloud_fraction() - 0.20) < 2.0 / sc.ncol
    # in-cloud extinction: the rank map onto lognormal(median 0.03, sigma 0.8)
    v = sc.k_cld[sc.k_cld > 0].astype(np.float64)
    assert np.median(v) == pytest.approx(0.03, rel=1e-3)
    assert np.std(np.log(v)) == pytest.approx(0.8, rel=5e-3)
    cloudy = sc.k_cld > 0
    assert np.all(sc.ssa_cld[cloudy] == np.float32(0.999999)) and np.all(sc.g_cld[cloudy] == np.float32(0.86))
    # bases U(700, 1000) m, centres 2 sigma_z (<= 600 m) above, 3 sigma_z boxes
    lo, hi = _cloud_heights(sc)
    assert lo >= 700.0 and hi <= 1000.0 + 5 * 300.0
    assert sc.albedo.min() >= 0.15 and sc.albedo.max() <= 0.25


def test_cumulus_benchmark_scene_optical_depths():
    """The figures quoted for the benchmark scene (seed 1): mean cloudy-column
    optical depth ~13, largest ~150, cloud layer 0.8-1.8 km."""
    sc = scenes.cumulus_scene(seed=1)
    tau = (sc.k_cld.astype(np.float64) * sc.dz).sum(axis=0)
    assert 12.0 < tau[tau > 0].mean() < 14.0 and 140.0 < tau.max() < 160.0
    lo, hi = _cloud_heights(sc)
    assert 800.0 <= lo and hi <= 1800.0


def test_generators_are_seeded():
    a, b = scenes.cumulus_scene(seed=7, nx=64, ny=64, nz=64), scenes.cumulus_scene(seed=7, nx=64, ny=64, nz=64)
    c = scenes.cumulus_scene(seed=8, nx=64, ny=64, nz=64)
    assert all(np.array_equal(x, y) for x, y in zip((*a.fields(), a.albedo), (*b.fields(), b.albedo)))
    assert not np.array_equal(a.k_cld, c.k_cld)


def test_gpoint_table_and_batch_scenes():
    scale, flux = scenes.gpoint_table()
    assert scale.shape == flux.shape == (112,)
    assert scale.min() >= 1e-3 and scale.max() <= 10.0 and scale.max() / scale.min() > 1e3
    assert flux.sum() == pytest.approx(1000.0) and flux.max() / flux.min() <= 10.0 + 1e-9
    shapes = [(s.nx, s.ny, s.nz) for s in scenes.batch_scenes()]
    assert shapes == [(128, 128, 96), (192, 96, 128), (256, 256, 128), (64, 64, 64)]
