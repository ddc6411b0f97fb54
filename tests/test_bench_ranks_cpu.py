"""The multi-rank path of bench.py on CPU: two gloo ranks (the replicas
layout of `bench.py --gpus 2`), each reporting its own elapsed time; every
rank must see the maximum over ranks after the reduction, and the barrier
must order the ranks.  No GPU and no library call is involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    torch.cuda.is_available = lambda: False  # CPU ranks: gloo even on a GPU machine
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (ws, rank, rank)
    elapsed = 10.0 + 5.0 * rank  # rank 1 is the slow one
    bench.barrier(w)
    m = bench.max_over_ranks(elapsed, w, torch.device("cpu"))
    # the whole-job value uses the slowest rank's time
    value = 30 * w / (m / 1e3)
    out.put((rank, m, value))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not available")
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(ws))
    assert [g[1] for g in got] == [15.0, 15.0]
    assert got[0][2] == got[1][2] == 30 * 2 / 0.015
