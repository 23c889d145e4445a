"""The multi-rank path of bench.py on the CPU (gloo, two ranks): each rank runs
its own instance (its own seed), and rank 0 reports the slowest rank's time and
the particle-steps of all ranks.  No GPU, no collective on the data path."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1511_08225_gb300 import inputs
    # per-rank timing and work differ; the instances are seeded by rank
    ms = 10.0 + 5.0 * rank
    ps = 1000.0 * (rank + 1)
    t, total = bench.aggregate_ranks(ms, ps, dist, "cpu")
    prob = bench.make_problem(inputs.SEED + rank)
    st = inputs.load_state(dict(prob, n_cells=8, species=[dict(sp, ppc=4) for sp in prob["species"]]))
    out.put((rank, t, total, float(st[0][2][0, 0])))
    dist.destroy_process_group()


def test_two_ranks_report_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, t, total, _ in res:
        assert t == pytest.approx(15.0) and total == pytest.approx(3000.0)
    # independent instances: the ranks' loads differ
    assert res[0][3] != res[1][3]
