"""GPU test of the double-buffered host pipeline: overlapping the copies with
the neighbouring steps' transport changes no result."""
import numpy as np
import pytest

from paper_2208_05247_b300 import pipeline, rt, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_pipelined_steps_equal_sequential_calls(small_scene):
    sc = small_scene
    N = 64 * sc.ncol
    steps = []
    for q, scale in enumerate((1.0, 2.0, 0.5, 1.5)):
        s = scenes.Scene("s%d" % q, sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, sc.k_gas, sc.ssa_gas,
                         (sc.k_cld * np.float32(scale)).astype(np.float32), sc.ssa_cld, sc.g_cld, sc.albedo)
        steps.append((s, 20.0 + 10 * q, 100 + q))
    want = []
    with rt.Tracer.from_scene(sc, 4, 4, 4) as t:
        for s, sza, seed in steps:
            t.set_optics(*s.fields())
            t.set_surface(s.albedo)
            t.build_accel(4, 4, 4)
            t.reset()
            t.trace(sza, 10.0, 1000.0, N, seed)
            f = t.fields()
            f["hr"] = t.heating_rate()
            want.append(f)
    t = rt.Tracer.from_scene(sc, 4, 4, 4)
    pipe = pipeline.HostPipeline(t, (4, 4, 4))
    outs = []
    for s, sza, seed in steps:
        fields = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in s.fields()]
        alb = torch.from_numpy(s.albedo).pin_memory()
        out = {k: torch.empty(sc.ncell if k in ("abs3d", "hr") else sc.ncol, dtype=torch.float64).pin_memory()
               for k in pipeline.OUT_KEYS}
        pipe.submit(fields, alb, sza, 10.0, 1000.0, N, seed, out)
        outs.append((out, fields, alb))          # keep the pinned inputs alive until the copies ran
    pipe.synchronize()
    t.close()
    for (out, _, _), w in zip(outs, want):
        for k in pipeline.OUT_KEYS:
            got = out[k].numpy().reshape(w[k].shape)
            scale = np.abs(w[k]).max()
            assert np.allclose(got, w[k], rtol=1e-12, atol=1e-12 * scale), k
