"""GPU tests of the diffuse share of the top boundary and of the paper's own
optics inputs (total extinction, cloud extinction, one albedo, g), Sec. 2.3."""
import numpy as np
import pytest

import oracle
from paper_2208_05247_b300 import rt, scenes
from tests import refs

pytestmark = pytest.mark.gpu

FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")


def test_gpu_diffuse_fraction_empty_atmosphere_and_absorbing_slab():
    sc = scenes.layered_scene(4, 4, 3, 50.0, 50.0, 100.0, k_gas=0.0, ssa_gas=0.0)
    f, N = 0.3, 2_000_000
    with rt.Tracer.from_scene(sc, 1, 1, 1) as t:
        t.trace(40.0, 0.0, 1000.0, N, 3, diffuse_fraction=f)
        fl = t.fields()
    F = 1000.0 * np.cos(np.deg2rad(40.0))
    se = F * np.sqrt(f * (1 - f) / N)
    assert abs(fl["sfc_dif"].mean() - f * F) < 4 * se
    # every photon lands; weights are scaled to energy in FP32 when tallied
    assert np.isclose(fl["sfc_dif"].mean() + fl["sfc_dir"].mean(), F, rtol=1e-6)
    k = np.array([1e-3, 3e-3], dtype=np.float32)
    dz = 150.0
    slab = scenes.layered_scene(3, 3, 2, 100.0, 100.0, dz, k_gas=k, ssa_gas=0.0)
    tau = float(np.sum(k.astype(np.float64)) * dz)
    p = 2 * refs.e3(tau)
    vals = []
    with rt.Tracer.from_scene(slab, 1, 1, 1) as t:
        for s in range(8):
            t.reset()
            t.trace(20.0, 0.0, 1.0, 500_000, 100 + s, diffuse_fraction=1.0)
            fl = t.fields()
            assert np.all(fl["sfc_dir"] == 0)
            vals.append(fl["sfc_dif"].mean() / np.cos(np.deg2rad(20.0)))
    v = np.array(vals)
    assert abs(v.mean() - p) < 4 * v.std(ddof=1) / np.sqrt(v.size) + 1e-12, (v.mean(), p)


def test_gpu_diffuse_fraction_parity_with_oracle(small_scene):
    B, N, f = 8, 2 ** 18, 0.4
    g = {k: [] for k in FIELDS}
    with rt.Tracer.from_scene(small_scene) as t:
        for s in range(B):
            t.reset()
            t.trace(50.0, 45.0, 800.0, N, 20 + s, diffuse_fraction=f)
            fl = t.fields(split=True)
            for k in FIELDS:
                g[k].append(fl[k])
    o = {k: [] for k in FIELDS}
    for s in range(B):
        r = oracle.trace(small_scene, 50.0, 45.0, 800.0, N, 400 + s, diffuse_fraction=f)
        for k in FIELDS:
            o[k].append(getattr(r, k))
    for k in FIELDS:
        rel, se = refs.domain_compare(np.stack(g[k]), np.stack(o[k]))
        assert abs(rel) < 4 * se + 1e-12, (k, rel, se)


def test_gpu_paper_optics_inputs(small_scene):
    """Total extinction, cloud extinction, one albedo and g: the same physics as
    the five-field inputs with k_gas = k_ext - k_cld and equal albedos."""
    sc = small_scene
    k_ext = (sc.k_gas + sc.k_cld).astype(np.float32)
    k_c = sc.k_cld
    w = np.where(sc.k_cld > 0, np.float32(0.9999), np.float32(0.9)).astype(np.float32)
    eq = scenes.Scene("equivalent", sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, (k_ext - k_c).astype(np.float32),
                      w, k_c, w, sc.g_cld, sc.albedo)
    B, N = 8, 2 ** 18
    g = {k: [] for k in FIELDS}
    with rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz) as t:
        rt.rt_set_optics_total(t.h, t.ncell, k_ext, k_c, w, sc.g_cld)
        t.set_surface(sc.albedo)
        t.build_accel()
        for s in range(B):
            t.reset()
            t.trace(30.0, 0.0, 1000.0, N, 60 + s)
            fl = t.fields(split=True)
            for k in FIELDS:
                g[k].append(fl[k])
        bad = k_c.copy()
        bad[0, 0, 0] = k_ext[0, 0, 0] + 1.0            # cloud extinction above the total
        with pytest.raises(rt.RtError):
            rt.rt_set_optics_total(t.h, t.ncell, k_ext, bad, w, sc.g_cld)
    o = {k: [] for k in FIELDS}
    for s in range(B):
        r = oracle.trace(eq, 30.0, 0.0, 1000.0, N, 800 + s)
        for k in FIELDS:
            o[k].append(getattr(r, k))
    for k in FIELDS:
        rel, se = refs.domain_compare(np.stack(g[k]), np.stack(o[k]))
        assert abs(rel) < 4 * se + 1e-12, (k, rel, se)


def test_batch_job_with_diffuse_fraction(small_scene):
    t = rt.Tracer(small_scene.nx, small_scene.ny, small_scene.nz, small_scene.dx, small_scene.dy, small_scene.dz)
    t.set_options(batch_optics=1)
    t.set_optics(*small_scene.fields())
    t.set_surface(small_scene.albedo)
    t.build_accel()
    rt.rt_trace_batch([dict(scene=t, sza_deg=30.0, toa_flux=1000.0, gas_scale=1.0, photons=400_000,
                            diffuse_fraction=1.0)], seed=5)
    fl = t.fields()
    assert np.all(fl["sfc_dir"] == 0) and fl["sfc_dif"].sum() > 0
    t.close()
