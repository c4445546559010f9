"""The replica path of bench.py (N > 1 ranks) on CPU: world_size 2 over gloo.

Each rank solves its own right-hand side; the whole-job throughput is the sum of the units of
all ranks over the slowest rank's time.  No data-path collective exists; only these reductions."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    units = 1000.0 * (rank + 1)          # rank r processed (r+1) thousand unknown-iterations
    ms = 10.0 * (rank + 1)               # and took (r+1) * 10 ms
    val, ms_max, units_all = bench.replica_throughput(units, ms, ws, device="cpu")
    bench.barrier(ws)
    q.put((rank, val, ms_max, units_all))
    dist.destroy_process_group()


def test_replica_reductions_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, val, ms_max, units_all in res:
        assert ms_max == 20.0
        assert units_all == 3000.0
        assert val == pytest.approx(3000.0 / 0.020)
