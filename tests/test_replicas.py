"""bench.py --gpus N runs N independent replicas (no collective on the data path):
the host-side rank logic, checked with two gloo processes on the CPU.

* the step time is the maximum over ranks (every rank receives it);
* the barrier brackets the timed region on every rank;
* the reference arm (the oracle) runs on rank 0 only: other ranks return at once
  without work or output.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup(None)
    d = bench.dist_init(w, "gloo")
    bench.dist_barrier(d)
    m = bench.dist_max(d, 10.0 * (rank + 1), "cpu")
    bench.dist_barrier(d)
    # the reference arm: rank 0 alone does the work
    ran = None
    if rank != 0:
        class A:
            pass
        ran = bench.run_reference(A())  # returns before touching any argument
    q.put((r, w, m, ran))
    d.destroy_process_group()


def test_two_replicas_max_and_barrier():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[2] == 20.0 for o in out)      # max over ranks, on every rank
    assert out[1][3] is None                    # rank 1 of the reference arm: no work


def test_single_process_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.dist_init(1, "gloo") is None
    assert bench.dist_max(None, 3.5, "cpu") == 3.5
