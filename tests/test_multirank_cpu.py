"""Multi-rank paths on CPU (gloo, world size 2): the benchmark's reduction over ranks
(slowest rank's time, every rank's work), and sharding one update's primaries over
ranks by ray range -- each rank traces [r N/W, (r+1) N/W) with first_ray, and the
primary-weighted sum of the ranks' IRs equals the single-process trace (the oracle
stands in for the GPU path, which this machine cannot run)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, ws, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)


def _reduce_worker(rank, ws, port, out):
    _init(rank, ws, port)
    import bench
    t, w = bench.reduce_over_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), "cpu")
    out[rank] = (t, w)
    dist.destroy_process_group()


def _shard_worker(rank, ws, port, out):
    _init(rank, ws, port)
    import oracle
    from paper_1803_00430_gb300 import scenes
    sc = scenes.shoebox(bands=4)
    osc = oracle.OracleScene(sc.verts, sc.tris, sc.tri_material, sc.absorption, sc.scattering)
    N = 600
    per = N // ws
    p = oracle.TraceParams(num_rays=per, first_ray=rank * per, seed=77, max_order=12, sh_order=1, num_bins=400,
                           min_order=1, ir_rate_hz=1000.0)
    H, st, _ = oracle.trace(osc, p, sc.listener, sc.sources)
    part = torch.tensor(H * st["primaries"], dtype=torch.float64)
    k = torch.tensor([float(st["primaries"])], dtype=torch.float64)
    dist.all_reduce(part)
    dist.all_reduce(k)
    out[rank] = (part / k).numpy()
    dist.destroy_process_group()


def _spawn(fn, ws=2):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(fn, args=(ws, port, out), nprocs=ws, join=True)
        return dict(out)


def test_bench_reduction_over_ranks():
    out = _spawn(_reduce_worker)
    for r in range(2):
        assert out[r] == (15.0, 300.0)


def test_ray_range_sharding_equals_single_trace():
    import oracle
    from paper_1803_00430_gb300 import scenes
    out = _spawn(_shard_worker)
    sc = scenes.shoebox(bands=4)
    p = oracle.TraceParams(num_rays=600, seed=77, max_order=12, sh_order=1, num_bins=400, min_order=1,
                           ir_rate_hz=1000.0)
    osc = oracle.OracleScene(sc.verts, sc.tris, sc.tri_material, sc.absorption, sc.scattering)
    H, st, _ = oracle.trace(osc, p, sc.listener, sc.sources)
    assert np.abs(H).max() > 0
    for r in range(2):
        np.testing.assert_allclose(out[r], H, rtol=1e-12, atol=1e-15 * np.abs(H).max())
