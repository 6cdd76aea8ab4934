"""rt_trace_noalloc: tracing for callers that cannot allocate device memory.

An atmospheric model that reserves its whole GPU memory pool at start-up, or a
framework whose allocator must own every device buffer, cannot hold an
rt_handle (rt_create allocates). rt_trace_noalloc lets such a caller trace with
its own buffers only. These tests check that it reproduces rt_trace on the same
seed, on two calls in a row (the calls share one fixed scratch array, which
must be cleared correctly each time), and that grids whose majorant would not
fit that array are rejected with a clear error.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2208_05247_b300 import build, rt, scenes


def test_noalloc_rejects_a_majorant_larger_than_its_fixed_scratch():
    build.build()
    lib = rt.library()
    dummy = np.zeros(4, np.float64)        # never touched: the call fails before any device work
    p = dummy.ctypes.data
    # 2048 x 1024 x 512 cells at coarsening 1 need 2^30 coarse cells > 2^20
    rc = lib.rt_trace_noalloc(2048, 1024, 512, 1.0, 1.0, 1.0, p, p, p, p, p, p, 1, 1, 1, 30.0, 0.0, 1000.0,
                              10, 1, p, p, p, p, p, None, None)
    assert rc == rt.RT_E_INVAL
    assert "coarse cells exceed the fixed maximum" in rt.rt_last_error()
    rc = lib.rt_trace_noalloc(32, 32, 32, 1.0, 1.0, 1.0, p, p, p, p, p, p, 0, 0, 0, 95.0, 0.0, 1000.0,
                              10, 1, p, p, p, p, p, None, None)
    assert rc == rt.RT_E_INVAL


@pytest.mark.gpu
def test_noalloc_matches_rt_trace_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    sc = scenes.ellipsoid_scene(seed=0)
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in sc.fields()]
    alb = torch.from_numpy(sc.albedo).to(dev)
    N = 300_000
    outs = {k: torch.zeros(n, dtype=torch.float64, device=dev)
            for k, n in (("abs_dir", sc.ncell), ("abs_dif", sc.ncell), ("sfc_dir", sc.ncol),
                         ("sfc_dif", sc.ncol), ("toa_up", sc.ncol))}
    for call, seed in enumerate((41, 42)):
        # the existing entry point, through a handle
        with rt.Tracer.from_scene(sc, 4, 4, 4) as t:
            t.trace(30.0, 0.0, 1000.0, N, seed)
            ref = t.fields(split=True)
            ref_events = t.stats()["events"]
        for v in outs.values():
            v.zero_()
        events = rt.rt_trace_noalloc(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, *ins, alb, 30.0, 0.0, 1000.0, N,
                                     seed, outs["abs_dir"], outs["abs_dif"], outs["sfc_dir"], outs["sfc_dif"],
                                     outs["toa_up"], coarse=(4, 4, 4))
        torch.cuda.synchronize()
        assert events == ref_events, (call, events, ref_events)
        for k, v in outs.items():
            got = v.cpu().numpy().reshape(ref[k].shape)
            scale = np.abs(ref[k]).max()
            assert np.allclose(got, ref[k], rtol=1e-12, atol=1e-12 * scale), (call, k)
