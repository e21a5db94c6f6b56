"""A job split over two processes on the CUDA path (Sec. 2.3.3: independent
batches, jobs split over GPUs), world size 2 over gloo.

Each process runs psl_run on its own history range of one plan (the one
GPU of this machine stands in for each rank's GPU: the ranks' kernels never
wait on one another, only the host all-reduce joins them), sums the ranks'
int64 tallies with engine.reduce_tallies, and reads out one dose.  The
summed tally and ledger must equal a single-process run of the whole range
bit for bit, and so must the dose.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_HIST = 200_000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload():
    from paper_1302_1861_b300 import inputs
    w = inputs.config1(n_records=20_000, n_histories=N_HIST)
    w.n_batches = 4
    return w


def _run(rank, world, group=None):
    """This rank's shard of the plan, reduced over the ranks when world > 1;
    returns (raw tallies + ledger, dose) as host arrays."""
    import torch

    from paper_1302_1861_b300 import capi, engine
    w = _workload()
    dw = engine.upload(w)
    first, n, n_plan = engine.shard_histories(rank, world, N_HIST // world)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, n_plan, w.seed)
    tally = capi.psl_tally_create(dw.phantom, w.n_batches)
    capi.psl_run(plan, dw.phantom, capi.physics(), tally, first, n)
    if world > 1:
        engine.reduce_tallies(tally, group)
    nvox = dw.mat_t.numel()
    dose = torch.empty(nvox, dtype=torch.float64, device="cuda")
    sigma = torch.empty_like(dose)
    lg = torch.empty(3, dtype=torch.float64, device="cuda")
    capi.dose_readout(tally, dw.phantom, engine.normalisation(plan, n_plan), dose, sigma, lg)
    t, ledger = engine.tally_views(tally)
    raw = np.concatenate([t.cpu().numpy(), ledger.cpu().numpy()])
    out = raw, dose.cpu().numpy(), sigma.cpu().numpy()
    tally.close(); plan.close(); store.close()
    return out


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    raw, dose, sigma = _run(rank, world)
    np.save(os.path.join(out_dir, f"raw{rank}.npy"), raw)
    np.save(os.path.join(out_dir, f"dose{rank}.npy"), dose)
    np.save(os.path.join(out_dir, f"sigma{rank}.npy"), sigma)
    dist.barrier()
    dist.destroy_process_group()


def test_two_process_reduce_equals_single_process(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    raw, dose, sigma = _run(0, 1)
    assert raw[:-12].sum() > 0
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"raw{r}.npy"), raw), r
        assert np.array_equal(np.load(tmp_path / f"dose{r}.npy"), dose), r
        assert np.array_equal(np.load(tmp_path / f"sigma{r}.npy"), sigma), r
