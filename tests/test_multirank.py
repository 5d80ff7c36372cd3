"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
max-over-ranks timing, the whole-job sum of work, the barrier, and the
per-rank Philox stream tags (replicas never share a random stream)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = bench.dist_info()
    bench.barrier(w)
    mx = bench.reduce_max(10.0 * (rank + 1), w)
    sm = bench.reduce_sum(1.5 + rank, w)
    tags = [bench.stream_tag(rank, p) for p in range(4)]
    q.put((r, w, mx, sm, tags))
    dist.destroy_process_group()


def test_two_rank_reductions_and_stream_tags():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 20.0 for o in out)       # max over ranks
    assert all(o[3] == 1.5 + 2.5 for o in out)  # whole-job sum
    tags = [t for o in out for t in o[4]]
    assert len(set(tags)) == len(tags)          # disjoint random streams across replicas
