"""Host-side logic of the multi-rank benchmark path, on CPU with the gloo backend
(world size 2): max-over-ranks timing, whole-job throughput and the partition of an
ensemble's fields over ranks.  The single-field step does not shard (independent
replicas, no collective on the data path); the ensemble shards by fields."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [0.25, 0.75][rank]
    m = bench.max_over_ranks(secs)
    v = bench.job_value(1_048_576, 100, world, m)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, v = out[r]
        assert m == 0.75
        assert v == pytest.approx(1_048_576 * 100 * 2 / 0.75 / 1e9)


def test_single_process_is_identity():
    assert bench.max_over_ranks(1.5) == 1.5


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_fields_covers_every_field_once_and_balances(world):
    from paper_1407_1309_gb300 import workloads
    import numpy as np
    rng = np.random.default_rng(0)
    sizes = [int(n) ** 2 for n in rng.choice(np.arange(64, 513, 32), size=512)]
    parts = bench.partition_fields(sizes, world)
    assert sorted(f for p in parts for f in p) == list(range(512))
    loads = [sum(sizes[f] for f in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
