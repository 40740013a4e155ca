"""The replica path of `bench.py --gpus N` on CPU with two gloo ranks: the job
time is the slowest rank's and the pairs are summed over ranks."""
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2])
def test_replicas_aggregate_over_gloo_ranks(world):
    import _replica_worker

    times = [1.5, 2.25, 0.75, 3.0][:world]
    pairs = [1e11, 3e11, 5e11, 7e11][:world]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker.run, args=(r, world, port, times, pairs, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, p in out:
        assert t == max(times)
        assert p == sum(pairs)


def test_single_rank_is_identity():
    from paper_2107_02010_gb300 import replicas

    assert replicas.aggregate(1.25, 7.0, "cpu") == (1.25, 7.0)
