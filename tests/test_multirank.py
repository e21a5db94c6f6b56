"""History-range sharding across ranks (world size 2, gloo, CPU).

Each rank computes the tally of its own history range of one plan with the
oracle; the product's int64 rank reduce (engine.sum_over_ranks, the step
engine.reduce_tallies runs on a tally's device arrays) over gloo must give
exactly the tally of the whole range computed in one process.  The same
reduce on the CUDA path's tallies is tests/test_gpu_multirank.py.  This is the multi-GPU contract of the
path: independent histories, random streams keyed by history id, integer
tallies, so any shard count gives bitwise-identical dose.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

N_HIST = 3000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload():
    from paper_1302_1861_b300 import inputs
    return inputs.config1(n_records=8000, n_histories=2 * N_HIST)


def _shard_tally(rank, world):
    import oracle
    from oracle import source
    from paper_1302_1861_b300 import engine
    w = _workload()
    first, n, n_plan = engine.shard_histories(rank, world, N_HIST * 2 // world)
    assert n_plan == w.n_histories
    st = source.psl_build(w.records, w.binning)
    pl = source.make_plan(st, w.beams, n_plan, w.seed, w.z_psl, w.sad)
    r = oracle.run_plan(w, n_histories=n, first=first, n_batches=1, nthreads=1, store=st, plan=pl)
    return r["tallies"][0], r["ledger"]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1302_1861_b300 import engine
    t, lg = _shard_tally(rank, world)
    tt = torch.from_numpy(np.ascontiguousarray(t.ravel()))
    tl = torch.from_numpy(np.ascontiguousarray(lg))
    engine.sum_over_ranks(tt, tl)           # the product's rank reduce, on host tensors here
    if rank == 0:
        np.save(out_path, np.concatenate([tt.numpy(), tl.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_partition_the_plan():
    from paper_1302_1861_b300 import engine
    seen = []
    for r in range(4):
        first, n, n_plan = engine.shard_histories(r, 4, 250)
        seen.extend(range(first, first + n))
        assert n_plan == 1000
    assert seen == list(range(1000))


def test_two_rank_gloo_sum_equals_single_process(tmp_path):
    out = str(tmp_path / "sum.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    whole, lg = _shard_tally(0, 1)
    expect = np.concatenate([whole.ravel(), lg])
    assert np.array_equal(got, expect)
    assert whole.sum() > 0
