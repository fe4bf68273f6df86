"""The multi-process host logic of bench.py on CPU (gloo, world size 2):
the job's time is the slowest rank's, every rank sees the same value, and
under torchrun the reference arm runs on rank 0 only (other ranks exit 0
without work or output). The data path has no collective (replicas)."""
import argparse
import contextlib
import io
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    slowest = bench.max_over_ranks(1.5 + rank)       # rank 1 is the slow one
    ws, r, local = bench.dist_env()
    out = io.StringIO()
    rc = None
    if rank == 1:
        args = argparse.Namespace(gpus=2, steps=1, warmup=3, workload=2)
        with contextlib.redirect_stdout(out):
            rc = bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, ws, r, rc, out.getvalue()))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2.5, 2.5]
    assert [(x[2], x[3]) for x in res] == [(2, 0), (2, 1)]
    assert res[1][4] == 0 and res[1][5] == ""
