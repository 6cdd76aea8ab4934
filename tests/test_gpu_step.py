"""GPU tests of the coupled-model step (rt_step_*): one CUDA-graph replay per
radiation call with optics updated in place between calls (Sec. 2.2: the tracer
runs every 60 s of model time), plus the horizontal homogenisation of the
"-hom" experiments (Sec. 2.4).

A replay runs the same kernels with the same arguments as the ordinary calls,
so for equal seeds it must reproduce them up to the order of the FP64 atomic
additions in the transport kernel (relative differences ~1e-15); event counts
match exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2208_05247_b300 import rt, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12
PPC = 64


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def outputs(sc):
    return {k: torch.zeros(n, dtype=torch.float64, device="cuda") for k, n in
            (("abs3d", sc.ncell), ("hr", sc.ncell), ("sfc_dir", sc.ncol), ("sfc_dif", sc.ncol), ("toa_up", sc.ncol))}


def host(out, sc):
    s3, s2 = (sc.nz, sc.ny, sc.nx), (sc.ny, sc.nx)
    return {k: v.cpu().numpy().reshape(s3 if v.numel() == sc.ncell else s2) for k, v in out.items()}


def ordinary(sc, sza, az, flux, photons, seed, coarse, total_optics=None, diffuse=0.0, **opts):
    """The same radiation call through rt_set_optics / rt_trace / rt_fields."""
    with rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz) as t:
        if opts:
            t.set_options(**opts)
        if total_optics is None:
            t.set_optics(*sc.fields())
        else:
            rt.rt_set_optics_total(t.h, t.ncell, *total_optics)
        t.set_surface(sc.albedo)
        t.build_accel(*coarse)
        t.reset()
        t.trace(sza, az, flux, photons, seed, diffuse_fraction=diffuse)
        f = t.fields()
        f["hr"] = t.heating_rate()
        return f, t.stats()


def assert_same(got, want, keys=("abs3d", "hr", "sfc_dir", "sfc_dif", "toa_up")):
    for k in keys:
        scale = np.abs(want[k]).max() + 1e-300
        assert np.allclose(got[k], want[k], rtol=RTOL, atol=RTOL * scale), (k, np.abs(got[k] - want[k]).max())


class StepRig:
    """A handle plus device inputs/outputs bound into one rt_step."""

    def __init__(self, sc, coarse=(4, 4, 4), homogenize=0, bind_albedo=True, **opts):
        self.sc = sc
        self.t = rt.Tracer.from_scene(sc, *coarse, **opts)
        self.inp = [dev(a) for a in sc.fields()]
        self.alb = dev(sc.albedo) if bind_albedo else None
        self.out = outputs(sc)
        self.photons = PPC * sc.ncol
        self.step = rt.rt_step_create(self.t.h, sc.ncell, sc.ncol, self.inp, self.photons, albedo=self.alb,
                                      homogenize=homogenize, **self.out)

    def launch(self, sza, az, flux, seed, diffuse=0.0):
        rt.rt_step_launch(self.step, sza, az, flux, diffuse, seed)
        rt.rt_synchronize(self.t.h)
        return host(self.out, self.sc), self.t.stats()

    def close(self):
        rt.rt_step_destroy(self.step)
        self.t.close()


def test_replay_equals_ordinary_calls_and_follows_updated_optics(small_scene):
    sc = small_scene
    rig = StepRig(sc)
    try:
        got, st = rig.launch(30.0, 20.0, 1000.0, 11)
        want, wst = ordinary(sc, 30.0, 20.0, 1000.0, rig.photons, 11, (4, 4, 4))
        assert st["events"] == wst["events"] and st["photons"] == rig.photons
        assert_same(got, want)
        # the energy ledger of the replay closes as an ordinary call's does
        lhs = st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
        rhs = st["energy_toa_up"] + st["energy_atm_abs"] + st["energy_sfc_abs"]
        assert st["energy_in"] == wst["energy_in"]
        assert abs(lhs - rhs) < 1e-9 * st["energy_in"]

        # the next model step: thicker clouds and a darker surface, written in place
        sc2 = scenes.Scene("step2", sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, sc.k_gas, sc.ssa_gas,
                           (sc.k_cld * np.float32(2.0)).astype(np.float32), sc.ssa_cld, sc.g_cld,
                           (sc.albedo * np.float32(0.5)).astype(np.float32))
        rig.inp[2].copy_(dev(sc2.k_cld))
        rig.alb.copy_(dev(sc2.albedo))
        got2, st2 = rig.launch(45.0, 200.0, 900.0, 12, diffuse=0.25)
        want2, wst2 = ordinary(sc2, 45.0, 200.0, 900.0, rig.photons, 12, (4, 4, 4), diffuse=0.25)
        assert st2["events"] == wst2["events"]
        assert_same(got2, want2)

        # back to the first state and seed: the first result again
        rig.inp[2].copy_(dev(sc.k_cld))
        rig.alb.copy_(dev(sc.albedo))
        got3, st3 = rig.launch(30.0, 20.0, 1000.0, 11)
        assert st3["events"] == st["events"]
        assert_same(got3, got)
    finally:
        rig.close()


def test_invalid_inputs_trace_nothing_and_the_next_step_recovers(small_scene):
    sc = small_scene
    rig = StepRig(sc)
    try:
        good, _ = rig.launch(30.0, 0.0, 1000.0, 3)
        k = rig.inp[2].clone()
        bad = k.clone()
        bad[5] = float("nan")
        rig.inp[2].copy_(bad)
        rt.rt_step_launch(rig.step, 30.0, 0.0, 1000.0, 0.0, 3)
        with pytest.raises(rt.RtError) as e:
            rt.rt_synchronize(rig.t.h)
        assert e.value.code == rt.RT_E_INVAL
        st = rig.t.stats()
        assert st["photons"] == 0 and st["events"] == 0 and st["status"] == rt.RT_E_INVAL
        assert all(float(v.abs().max()) == 0.0 for v in rig.out.values())
        # an albedo outside [0, 1] is caught the same way
        rig.inp[2].copy_(k)
        a = rig.alb.clone()
        rig.alb[0] = 1.5
        rt.rt_step_launch(rig.step, 30.0, 0.0, 1000.0, 0.0, 3)
        with pytest.raises(rt.RtError):
            rt.rt_synchronize(rig.t.h)
        rig.alb.copy_(a)
        again, st = rig.launch(30.0, 0.0, 1000.0, 3)
        assert st["status"] == 0 and st["photons"] == rig.photons
        assert_same(again, good)
    finally:
        rig.close()


def test_handle_belongs_to_its_step(small_scene):
    sc = small_scene
    rig = StepRig(sc, bind_albedo=False)
    try:
        for call in (lambda: rig.t.trace(30.0, 0.0, 1000.0, 1000, 1),
                     lambda: rig.t.set_optics(*sc.fields()),
                     lambda: rig.t.build_accel(2, 2, 2),
                     lambda: rig.t.set_options(block_size=128),
                     lambda: rt.rt_destroy(rig.t.h),
                     lambda: rt.rt_step_create(rig.t.h, sc.ncell, sc.ncol, rig.inp, 10)):
            with pytest.raises(rt.RtError) as e:
                call()
            assert e.value.code == rt.RT_E_STATE
        # without a bound albedo the handle's surface is used and may change between steps
        got, _ = rig.launch(20.0, 0.0, 1000.0, 5)
        rig.t.set_surface(np.zeros_like(sc.albedo))
        got0, _ = rig.launch(20.0, 0.0, 1000.0, 5)
        assert got0["toa_up"].sum() < got["toa_up"].sum()
        sc0 = scenes.Scene("black", sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, sc.k_gas, sc.ssa_gas, sc.k_cld,
                           sc.ssa_cld, sc.g_cld, np.zeros_like(sc.albedo))
        want0, _ = ordinary(sc0, 20.0, 0.0, 1000.0, rig.photons, 5, (4, 4, 4))
        assert_same(got0, want0)
    finally:
        rt.rt_step_destroy(rig.step)
    # once its step is destroyed the handle takes the ordinary calls again
    try:
        rig.t.set_optics(*sc.fields())
        rig.t.build_accel(2, 2, 2)
        rig.t.reset()
        rig.t.trace(30.0, 0.0, 1000.0, 1000, 1)
        rig.t.synchronize()
        assert rig.t.stats()["photons"] == 1000
    finally:
        rig.t.close()


@pytest.mark.parametrize("bits", [rt.RT_HOM_SURFACE, rt.RT_HOM_HEATING, rt.RT_HOM_SURFACE | rt.RT_HOM_HEATING])
def test_homogenised_outputs_are_layer_means(small_scene, bits):
    sc = small_scene
    plain = StepRig(sc)
    hom = StepRig(sc, homogenize=bits)
    try:
        p, _ = plain.launch(30.0, 228.1, 1000.0, 21)
        h, _ = hom.launch(30.0, 228.1, 1000.0, 21)
    finally:
        plain.close()
        hom.close()
    surf = ("sfc_dir", "sfc_dif")
    heat = ("abs3d", "hr")
    for k in surf + heat + ("toa_up",):
        on = (k in surf and bits & rt.RT_HOM_SURFACE) or (k in heat and bits & rt.RT_HOM_HEATING)
        want = oracle.homogenize(p[k]) if on else p[k]
        scale = np.abs(p[k]).max()
        assert np.allclose(h[k], want, rtol=RTOL, atol=RTOL * scale), k
    # homogenisation keeps the domain totals
    assert np.isclose(h["sfc_dir"].sum(), p["sfc_dir"].sum(), rtol=1e-12)
    assert np.isclose(h["abs3d"].sum(), p["abs3d"].sum(), rtol=1e-12)


def test_total_optics_and_fp32_tallies(small_scene):
    sc = small_scene
    k_ext = (sc.k_gas + sc.k_cld).astype(np.float32)
    w = np.where(sc.k_cld > 0, np.float32(0.9999), np.float32(0.9)).astype(np.float32)
    total = (k_ext, sc.k_cld, w, sc.g_cld)
    for prec in (rt.RT_TALLY_FP64, rt.RT_TALLY_FP32):
        t = rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz)
        t.set_options(tally_precision=prec)
        t.reset()
        rt.rt_set_optics_total(t.h, t.ncell, *total)
        t.set_surface(sc.albedo)
        t.build_accel(4, 4, 4)
        inp = [dev(a) for a in total]
        out = outputs(sc)
        step = rt.rt_step_create(t.h, sc.ncell, sc.ncol, inp, PPC * sc.ncol, optics=rt.RT_OPTICS_TOTAL, **out)
        try:
            rt.rt_step_launch(step, 35.0, 10.0, 1000.0, 0.0, 8)
            rt.rt_synchronize(t.h)
            got = host(out, sc)
        finally:
            rt.rt_step_destroy(step)
            t.close()
        want, _ = ordinary(sc, 35.0, 10.0, 1000.0, PPC * sc.ncol, 8, (4, 4, 4), total_optics=total,
                           tally_precision=prec)
        if prec == rt.RT_TALLY_FP64:
            assert_same(got, want)
        else:
            # FP32 atomics in a different order: agreement to FP32 accumulation error
            for k in want:
                scale = np.abs(want[k]).max()
                assert np.allclose(got[k], want[k], rtol=1e-3, atol=1e-4 * scale), k
