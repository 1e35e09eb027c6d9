"""The N > 1 path of the benchmark on CPU processes (gloo, world size 2):
every rank generates its own seeded image (independent problems, no data
exchange), and the whole-job figures are the slowest rank's time and the
units of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w = bench.make_workload("nuclei2d_small", rank)
    n_roi = int(len(np.unique(w.mask[w.mask > 0])))
    t_ms = 1.0 + 0.5 * rank  # stands in for this rank's measured step time
    t, n = bench.reduce_over_ranks(dist, "cpu", t_ms, n_roi)
    out.put((rank, n_roi, int(w.image.sum()), t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_independent_images_and_whole_job_figures():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, s0, t0, tot0), (r1, n1, s1, t1, tot1) = res
    assert s0 != s1                      # each rank has its own image
    assert t0 == t1 == 1.5               # slowest rank's time
    assert tot0 == tot1 == n0 + n1       # units of all ranks


def test_single_rank_passthrough():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(None, "cpu", 2.5, 7) == (2.5, 7)
