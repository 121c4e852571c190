"""Multi-process path of bench.py on CPU: two gloo ranks run replicas (no
data-path collective); the barrier, the max over ranks of the elapsed time
and the job rate (units of all ranks / slowest rank's time) are the only
collectives.  Runs without a GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    from paper_1406_7416_gb300.replicas import Replicas
    rep = Replicas("gloo")
    rep.barrier()
    slowest = rep.max_over_ranks(1.5 + rank)            # rank r "took" 1.5 + r seconds
    rate = rep.job_rate(100.0, 1.0 + rank)              # 100 units on every rank
    rep.close()
    out.put((rank, rep.world, slowest, rate))


def test_two_gloo_ranks_reduce_time_and_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, slowest, rate in res:
        assert world == 2
        assert slowest == pytest.approx(2.5)
        assert rate == pytest.approx(2 * 100.0 / 2.0)


def test_single_process_is_local(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1406_7416_gb300.replicas import Replicas
    rep = Replicas("gloo")
    assert rep.world == 1 and rep.max_over_ranks(3.0) == 3.0
    assert rep.job_rate(10.0, 2.0) == 5.0
    rep.close()
