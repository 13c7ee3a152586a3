"""Sharding and the final merge across ranks, on CPU with the gloo backend.

Each rank owns a contiguous block of global patient ids (weak scaling) and
produces its per-patient records; rank 0 gathers them in global-id order and
reduces once.  Here the records come from the oracle, so the test runs with no
GPU: the merged records must equal those of one run over all ids, and the
population summary of the merge must equal the single-run summary.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2202_13927_gb300 import dist as D


def test_shard_and_split_ranges():
    assert D.shard_range(0, 4, 100) == (0, 100)
    assert D.shard_range(3, 4, 100, base=7) == (307, 407)
    parts = [D.split_range(r, 3, 10) for r in range(3)]
    assert parts == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        D.shard_range(2, 2, 5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _records(first, n):
    from oracle import oracle as O
    from paper_2202_13927_gb300 import workloads as W
    pop = W.population(n, 77, first_patient=first)
    people = O.create_population(pop)
    st = O.simulate(pop, people, W.scenario(0, horizon_periods=96), {}, nthreads=2)["stats"]
    return st


def _worker(rank, world, port, n, q, strong):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, last = D.split_range(rank, world, n) if strong else D.shard_range(rank, world, n)
    st = _records(first, last - first)
    local = torch.from_numpy(st.view(np.uint8).copy())
    merged = D.gather_records(local, rank, world)
    if rank == 0:
        q.put(merged.numpy().tobytes())
    else:
        assert merged is None
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n,strong", [(2, 40, False), (3, 100, True)])
def test_gather_equals_single_run(world, n, strong):
    """Weak scaling (equal blocks of n per rank) on two ranks, and strong
    scaling (100 ids split 33 / 33 / 34) on three: the gather handles shards
    of unequal size."""
    from oracle import oracle as O
    from oracle import popstats as OP
    total = n if strong else world * n
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q, strong)) for r in range(world)]
    for p in procs:
        p.start()
    merged_bytes = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    merged = np.frombuffer(merged_bytes, dtype=O.STATS_DTYPE)
    whole = _records(0, total)
    assert merged.shape[0] == total
    assert merged.tobytes() == whole.tobytes()
    a = OP.population_stats(merged["tir"], merged["status"], merged["g_mean"], merged["g_min"],
                            merged["basal_u"], merged["bolus_u"], 96)
    b = OP.population_stats(whole["tir"], whole["status"], whole["g_mean"], whole["g_min"],
                            whole["basal_u"], whole["bolus_u"], 96)
    assert a["worst_patient"] == b["worst_patient"]
    np.testing.assert_array_equal(a["tir_quantile"], b["tir_quantile"])
