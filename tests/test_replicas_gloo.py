"""The N > 1 bench path is replicas with no data-path collective: each rank
encrypts its own stream (own key), the step time is the max over ranks, and the
rate counts the pixels of all ranks.  Exercised with world_size 2 on the gloo
backend on CPU (no GPU)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import synth

        key = synth.key_for_seed(0, bench.stream_seed(rank))
        # each rank's replica: its own stream, no exchange of frames or state
        X = synth.uniform_frames(1, 16, 16, 3, seed=5)
        Y = oracle.OracleCipher(0, key, 16, 16, 3, 4, 5).encrypt(X)
        slow = bench.reduce_max(1.0 + rank, "cpu")
        q.put((rank, key, Y.tobytes(), slow, bench.whole_job_rate(1_000_000, world, slow)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, k0, y0, s0, v0), (r1, k1, y1, s1, v1) = res
    assert k0 != k1 and y0 != y1          # independent streams
    assert s0 == s1 == 2.0                # max over ranks
    assert v0 == v1 == 2 * 1_000_000 / 2.0 / 1e6
