"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2): ranks label
disjoint frame sets (weak scaling, no data-path collective) and the job time is the max
over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2003_00575_gb300 import synth
    frames = 6
    seeds = list(range(bench.rank_first_seed(rank, frames),
                       bench.rank_first_seed(rank, frames) + frames))
    shapes = [synth.config_c4_frame(sd).range.shape for sd in seeds[:2]]
    every = [None] * world
    dist.all_gather_object(every, seeds)
    t = bench.reduce_max(dist, 10.0 + rank, torch.device("cpu"))
    q.put((rank, every, t, shapes))
    dist.destroy_process_group()


def test_two_ranks_disjoint_frames_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, every, t, shapes in out:
        assert t == 11.0                       # the slower rank decides
        a, b = set(every[0]), set(every[1])
        assert not (a & b) and len(a) == len(b) == 6
        assert all(len(s) == 2 for s in shapes)
