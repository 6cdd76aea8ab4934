"""Multi-rank sharding on CPU: two gloo ranks trace disjoint photon ranges of
one run (with the oracle as the tracer) and sum their tallies; the result
equals the single-process run exactly for integer counts."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_05247_b300 import shard


def test_ranges_cover_the_run_once():
    for world in (1, 2, 3, 7):
        per = 1001
        got = []
        for r in range(world):
            b, c, t = shard.photon_range(r, world, per)
            assert t == per * world
            got.extend(range(b, b + c))
        assert got == list(range(per * world))
        total = 10_007
        got = []
        for r in range(world):
            b, c, t = shard.split_range(r, world, total)
            got.extend(range(b, b + c))
        assert got == list(range(total))
    with pytest.raises(ValueError):
        shard.photon_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2208_05247_b300 import scenes
    sc = scenes.ellipsoid_scene(seed=0)
    begin, count, total = shard.photon_range(rank, world, 20_000)
    r = oracle.trace(sc, 30.0, 0.0, 1000.0, count, 77, id_begin=begin, photons_total=total, nthreads=2)
    t = [torch.from_numpy(r.counts[k].astype(np.int64).ravel()) for k in ("sfc_dir", "sfc_dif", "toa", "abs_dif")]
    shard.sum_tallies(t)
    if rank == 0:
        np.savez(out_path, *[x.numpy() for x in t])
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_run(tmp_path):
    import oracle
    from paper_2208_05247_b300 import scenes
    out = str(tmp_path / "sum.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    sc = scenes.ellipsoid_scene(seed=0)
    full = oracle.trace(sc, 30.0, 0.0, 1000.0, 40_000, 77)
    for i, k in enumerate(("sfc_dir", "sfc_dif", "toa", "abs_dif")):
        assert np.array_equal(got[f"arr_{i}"], full.counts[k].astype(np.int64).ravel()), k


def _fields_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2208_05247_b300 import scenes
    sc = scenes.ellipsoid_scene(seed=0)
    begin, count, total = shard.photon_range(rank, world, 15_000)
    # each rank normalises with the whole run's photon count (photons_total)
    r = oracle.trace(sc, 30.0, 0.0, 1000.0, count, 91, id_begin=begin, photons_total=total, nthreads=2)
    f = {k: torch.from_numpy(np.ascontiguousarray(getattr(r, k), dtype=np.float64)) for k in oracle.FIELDS}
    f["hr"] = torch.from_numpy(oracle.heating_rate(r.abs3d, sc.dz))
    shard.reduce_fields(f)
    if rank == 0:
        np.savez(out_path, **{k: v.numpy() for k, v in f.items()})
    dist.destroy_process_group()


def test_reduce_fields_gives_the_combined_run(tmp_path):
    """Three gloo ranks, normalised fields (W m^-2, W m^-3, K/day) summed with
    reduce_fields: the single run of all photons, to FP64 rounding."""
    import oracle
    from paper_2208_05247_b300 import scenes
    out = str(tmp_path / "fields.npz")
    mp.start_processes(_fields_worker, args=(3, _free_port(), out), nprocs=3, join=True, start_method="spawn")
    got = np.load(out)
    sc = scenes.ellipsoid_scene(seed=0)
    full = oracle.trace(sc, 30.0, 0.0, 1000.0, 45_000, 91)
    for k in oracle.FIELDS:
        want = getattr(full, k)
        assert np.allclose(got[k], want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), k
    hr = oracle.heating_rate(full.abs3d, sc.dz)
    assert np.allclose(got["hr"], hr, rtol=1e-12, atol=1e-12 * np.abs(hr).max())
