"""Host-side logic of bench.py, on CPU: algorithmic byte counts, launch counts,
and the multi-rank aggregation (max time, summed points) over a world_size-2
gloo process group (the replica path that bench.py --gpus N takes)."""
import os
import socket

import pytest

import bench
import workloads as W

torch = pytest.importorskip("torch")


def test_algorithmic_bytes_radial2d_256():
    spec, om, x, _ = W.make_workload("radial2d_256")
    ab = bench.algorithmic_bytes(spec)
    assert ab["interp"] == 8 * 512 * 512 + 206336 * (4 * 2 + 8 * 12 + 8)
    assert ab["gridding"] == ab["interp"]
    assert ab["scale_pad_fft"] == 8 * 256 * 256 + 8 * 512 * 512
    assert ab["ifft_crop_rescale"] == ab["scale_pad_fft"]


def test_launch_counts():
    assert bench.launches_per_step({"d": 2}, 10) == 2 + 1 + 1 + 1 + 2
    assert bench.launches_per_step({"d": 3}, 0) == 3 + 1 + 0 + 1 + 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    el, units = bench.reduce_over_ranks(1.0 + rank, 10.0 * (rank + 1), world)
    q.put((rank, el, units))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, el, units in res:
        assert el == 2.0 and units == 30.0


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(1.5, 7.0, 1) == (1.5, 7.0)
