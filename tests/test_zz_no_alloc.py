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


def test_noalloc_source_calls_no_allocator():
    """The entry point's file names no allocating CUDA call outside its comments
    (a later change that adds one would fail here, before any GPU run)."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(build.LIB), "csrc", "rt_noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", src)
    for name in ("cudaMalloc", "cudaMallocAsync", "cudaMallocManaged", "cudaMallocHost", "cudaFree", "cudaHostAlloc"):
        assert name not in code, name


def _noalloc_case(torch, sc, coarse, seeds, N=300_000):
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in sc.fields()]
    alb = torch.from_numpy(sc.albedo).to(dev)
    outs = {k: torch.zeros(n, dtype=torch.float64, device=dev)
            for k, n in (("abs_dir", sc.ncell), ("abs_dif", sc.ncell), ("sfc_dir", sc.ncol),
                         ("sfc_dif", sc.ncol), ("toa_up", sc.ncol))}
    for call, seed in enumerate(seeds):
        # the existing entry point, through a handle
        with rt.Tracer.from_scene(sc, *coarse) as t:
            t.trace(30.0, 0.0, 1000.0, N, seed)
            ref = t.fields(split=True)
            ref_events = t.stats()["events"]
        for v in outs.values():
            v.zero_()
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
        events = rt.rt_trace_noalloc(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, *ins, alb, 30.0, 0.0, 1000.0, N,
                                     seed, outs["abs_dir"], outs["abs_dif"], outs["sfc_dir"], outs["sfc_dif"],
                                     outs["toa_up"], coarse=coarse)
        torch.cuda.synchronize()
        # nothing was taken from torch's allocator (the call allocates nothing)
        assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == before
        assert events == ref_events, (coarse, call, events, ref_events)
        for k, v in outs.items():
            got = v.cpu().numpy().reshape(ref[k].shape)
            scale = np.abs(ref[k]).max()
            assert np.allclose(got, ref[k], rtol=1e-12, atol=1e-12 * scale), (coarse, call, k)


@pytest.mark.gpu
def test_noalloc_matches_rt_trace_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    _noalloc_case(torch, scenes.ellipsoid_scene(seed=0), (4, 4, 4), (41, 42))


@pytest.mark.gpu
@pytest.mark.parametrize("coarse", [(5, 3, 7), (0, 0, 0)])
def test_noalloc_ragged_and_default_coarse_grids(coarse):
    """Coarse cells that only partly cover the grid edge (5, 3, 7 on 32^3:
    boxes stay single cells there) and the default factors (0, 0, 0, the same
    default as rt_build_accel)."""
    torch = pytest.importorskip("torch")
    _noalloc_case(torch, scenes.ellipsoid_scene(seed=0), coarse, (43, 44), N=200_000)


@pytest.mark.gpu
def test_noalloc_rejects_invalid_optics_and_leaves_outputs_unchanged():
    torch = pytest.importorskip("torch")
    sc = scenes.ellipsoid_scene(seed=0)
    dev = torch.device("cuda", 0)
    kg = sc.k_gas.copy()
    kg[3, 4, 5] = np.nan
    ins = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (kg,) + sc.fields()[1:]]
    alb = torch.from_numpy(sc.albedo).to(dev)
    outs = [torch.zeros(n, dtype=torch.float64, device=dev) for n in (sc.ncell, sc.ncell, sc.ncol, sc.ncol, sc.ncol)]
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_noalloc(sc.nx, sc.ny, sc.nz, sc.dx, sc.dy, sc.dz, *ins, alb, 30.0, 0.0, 1000.0, 100_000, 7,
                            *outs, coarse=(4, 4, 4))
    assert e.value.code == rt.RT_E_INVAL
    assert all(float(o.abs().sum()) == 0.0 for o in outs)
    # the shared scratch recovers: the next valid call matches rt_trace again
    _noalloc_case(torch, sc, (4, 4, 4), (45,), N=100_000)
