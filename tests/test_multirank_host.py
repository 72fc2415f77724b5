"""Host logic of the multi-GPU (replicas, weak scaling) benchmark path, run as
two gloo ranks on the CPU: each rank steps its own seeded realisation, and the
reported time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    import seeded_inputs as si

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    seed = bench.shard_seed(0, rank)
    p = bench.workload(seed, "f32")
    pos = si.saw_chain(dict(p, n_beads=12), seed)
    t = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], dist, "cpu")
    q.put((rank, seed, t, pos[:, 0].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_realisations_and_reduce_max_time():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort()
    seeds = [o[1] for o in out]
    assert len(set(seeds)) == 2
    for o in out:
        assert o[2] == [2.0, 10.0, 0.5]
    assert not np.allclose(out[0][3], out[1][3])


def test_single_process_reduction_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.0], None, "cpu") == [3.0, 4.0]
