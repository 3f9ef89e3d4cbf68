"""The multi-GPU form is replicas: every rank decodes its own frames and the
only collective is the max-over-ranks of the timed region. This covers that
host logic with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    from paper_1505_01466_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    slow = bench.reduce_max(torch, 10.0 * (rank + 1), "cpu")       # the slowest rank sets the time
    _, frozen, fr = bench.make_code_inputs(bench.rank_seed(rank), 64)
    np.save(os.path.join(out_dir, f"llr{rank}.npy"), fr.llr_i8)
    np.save(os.path.join(out_dir, f"res{rank}.npy"),
            np.array([slow, bench.job_gbps(1691, 1 << 20, world, slow)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_max_time(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [np.load(tmp_path / f"res{r}.npy") for r in range(world)]
    for r in res:
        assert r[0] == 20.0                                  # max over ranks, seen by every rank
        assert r[1] == pytest.approx(1691 * (1 << 20) * 2 / 0.020 / 1e9)
    a, b = (np.load(tmp_path / f"llr{r}.npy") for r in range(world))
    assert a.shape == b.shape and not np.array_equal(a, b)   # each rank decodes different frames


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(torch, 3.25, "cpu") == 3.25
