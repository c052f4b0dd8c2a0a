"""Multi-process host logic of the replica runs (bench.py --gpus N), on CPU with
the gloo backend and world size 2: each rank times its own mock; the job's
throughput is all ranks' units over the slowest rank's time; seeds differ per
rank.  No GPU and no data-path collective is involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_2005_05328_gb300 import replicas as R
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = R.rank_info()
        R.barrier()
        units = 1000.0 * (rank + 1)
        secs = 2.0 + rank  # rank 1 is the slow one
        tot, tmax = R.aggregate(units, secs)
        q.put((r, w, lr, tot, tmax, R.throughput(tot, tmax), R.replica_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for o in out:
        assert o[3] == 3000.0 and o[4] == 3.0
        assert o[5] == pytest.approx(1000.0)
    assert out[0][6] != out[1][6]


def test_single_process_is_identity():
    from paper_2005_05328_gb300 import replicas as R
    assert R.aggregate(5.0, 2.0) == (5.0, 2.0)
    assert R.throughput(10.0, 2.0) == 5.0
