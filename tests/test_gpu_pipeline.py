"""GPU tests of the overlapped steps: the double-buffered host pipeline (with
one handle or two) and the ring of handles on device-resident inputs give the
fields of the same calls made one after the other."""
import numpy as np
import pytest

from paper_2208_05247_b300 import pipeline, rt, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _steps_and_sequential(sc, N):
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
    return steps, want


def _compare(got_list, want):
    for out, w in zip(got_list, want):
        for k in pipeline.OUT_KEYS:
            got = out[k].cpu().numpy().reshape(w[k].shape)
            scale = np.abs(w[k]).max()
            assert np.allclose(got, w[k], rtol=1e-12, atol=1e-12 * scale), k


@pytest.mark.parametrize("handles", [1, 2, 3])
def test_pipelined_steps_equal_sequential_calls(small_scene, handles):
    sc = small_scene
    N = 64 * sc.ncol
    steps, want = _steps_and_sequential(sc, N)
    ts = [rt.Tracer.from_scene(sc, 4, 4, 4) for _ in range(handles)]
    pipe = pipeline.HostPipeline(ts, (4, 4, 4))
    outs = []
    for s, sza, seed in steps:
        fields = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in s.fields()]
        alb = torch.from_numpy(s.albedo).pin_memory()
        out = {k: torch.empty(sc.ncell if k in ("abs3d", "hr") else sc.ncol, dtype=torch.float64).pin_memory()
               for k in pipeline.OUT_KEYS}
        pipe.submit(fields, alb, sza, 10.0, 1000.0, N, seed, out)
        outs.append((out, fields, alb))          # keep the pinned inputs alive until the copies ran
    pipe.synchronize()
    for t in ts:
        t.close()
    _compare([o for o, _, _ in outs], want)


def test_step_ring_equals_sequential_calls(small_scene):
    """Two handles on two streams, each step's fields copied out on its
    handle's stream before that handle's next step reuses the buffers."""
    sc = small_scene
    N = 64 * sc.ncol
    steps, want = _steps_and_sequential(sc, N)
    dev = torch.device("cuda")
    ts = [rt.Tracer(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz) for _ in range(2)]
    ring = pipeline.StepRing(ts, (4, 4, 4))
    main = torch.cuda.current_stream()
    inputs = [([torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in s.fields()],
               torch.from_numpy(s.albedo).to(dev)) for s, _, _ in steps]
    ring.wait_on(main)
    got, used = [], []
    for (s, sza, seed), (f, alb) in zip(steps, inputs):
        snap = {}
        j, _ = ring.submit(f, alb, sza, 10.0, 1000.0, N, seed,
                           after=lambda st, o, snap=snap: snap.update({k: v.clone() for k, v in o.items()}))
        got.append(snap)
        used.append(j)
    ring.join(main)
    torch.cuda.synchronize()
    assert used == [0, 1, 0, 1]
    for t in ts:
        assert t.stats()["status"] == 0
        t.close()
    _compare(got, want)

