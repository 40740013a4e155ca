"""Rank body of tests/test_replicas_gloo.py (a module of its own so that spawned
processes can import it)."""
import os


def run(rank, world, port, times, pairs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    from paper_2107_02010_gb300 import replicas

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, p = replicas.aggregate(times[rank], pairs[rank], torch.device("cpu"))
        dist.barrier()
        q.put((rank, t, p))
    finally:
        dist.destroy_process_group()
