"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): one map per rank, no
data-path collective, and the whole-job numbers taken as the slowest rank's time and the
sum of all ranks' site updates.  Also checks that each rank draws its own inputs."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: a slower device time and its own update count
    times, ups = bench.reduce_over_ranks([10.0 + 5.0 * rank, 20.0 - rank], [100 + rank, 200 * (rank + 1)], dist)
    out.put((rank, times, ups))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_numbers_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, ups in res:
        assert times == [15.0, 20.0]                    # max over ranks
        assert ups == [201.0, 600.0]                    # sum over ranks


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.5], [3, 4]) == ([1.5, 2.5], [3.0, 4.0])


@pytest.mark.slow
def test_each_rank_fills_its_own_map():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_1811_01604_gb300 import synth
    # the bench grid generator takes the rank as seed offset (checked on small masks)
    m0 = synth.mask_disks(128, 128, 0.5, 1_000_003 + 0)
    m1 = synth.mask_disks(128, 128, 0.5, 1_000_003 + 1)
    assert not np.array_equal(m0, m1)
    assert "seed_offset" in bench.make_inputs.__code__.co_varnames
