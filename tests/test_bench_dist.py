"""Multi-process logic of bench.py on the CPU (gloo, world size 2): replicas only.

Rank 0 builds the operator (or finds it in the on-disk cache) while rank 1 waits at a barrier and
then reads the same cached buffer; the step time reported is the maximum over ranks.  No data
moves between ranks (the right-hand sides are independent), so the only collectives are the
barrier and the max-reduction of the time."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, cache, q):
    os.environ.update({"WORLD_SIZE": "2", "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "FIO_CACHE": cache})
    sys.path.insert(0, ROOT)
    import argparse
    import hashlib

    import bench
    ws, r, _ = bench.dist_init()
    a = argparse.Namespace(kind="ex1", n=256, eps_bf=1e-6, eps_hif=1e-5)
    buf, info = bench.get_operator(a, r, ws)
    m = bench.allmax(ws, 10.0 + r)
    bench.barrier(ws)
    q.put((r, ws, hashlib.sha256(buf).hexdigest(), m, info["N"]))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replicas_share_the_operator_and_reduce_the_time(tmp_path):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, str(tmp_path), q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, h0, m0, n0), (r1, ws1, h1, m1, n1) = res
    assert (r0, r1, ws0, ws1) == (0, 1, 2, 2)
    assert h0 == h1            # the same factors on both replicas
    assert m0 == m1 == 11.0    # the step time is the max over ranks
    assert n0 == n1 == 256
