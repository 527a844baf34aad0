"""The benchmark's multi-rank host logic with world_size 2 over gloo on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.5, 4.25][rank]
        slowest = bench.max_over_ranks(local, world, "cpu")
        out.put((rank, slowest, bench.whole_job_rate(100.0, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [4.25, 4.25]
    assert got[0][2] == pytest.approx(200.0 / 4.25)


def test_reference_arm_prints_once_under_two_ranks():
    env_base = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    outs = []
    for rank in (0, 1):
        env = dict(env_base, RANK=str(rank), LOCAL_RANK=str(rank))
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                            "--steps", "1", "--warmup", "0", "--ref-iterations", "2"],
                           env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    line = json.loads(outs[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert outs[1] == ""


def test_shards_partition_the_workload():
    """Every item of a batch or request stream goes to exactly one rank, for any world
    size; contiguous blocks differ in size by at most one and come in rank order."""
    sys.path.insert(0, ROOT)
    from paper_2002_11710_gb300 import shard

    for n in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 4, 8):
            blocks = [shard.contiguous(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
            dealt = sorted(i for r in range(world) for i in shard.strided(n, r, world))
            assert dealt == list(range(n))
    with pytest.raises(ValueError):
        shard.contiguous(5, 2, 2)


def _shard_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_2002_11710_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.contiguous(1024, rank, world)
        mine = np.arange(lo, hi)
        stream = np.array(list(shard.strided(3001, rank, world)))
        all_batch = bench.gather_arrays(mine, world)
        all_stream = bench.gather_arrays(stream, world)
        total = bench.sum_over_ranks(len(mine), world, "cpu")
        out.put((rank, all_batch.tolist(), sorted(all_stream.tolist()), total))
    finally:
        dist.destroy_process_group()


def test_batch_and_stream_shards_gather_to_the_whole_gloo():
    """Under two gloo ranks, each rank's part of the 1,024-instance batch and of a
    request stream, gathered on the host, is the whole workload with no overlap."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, batch, stream, total in got:
        assert batch == list(range(1024))
        assert stream == list(range(3001))
        assert total == 1024
