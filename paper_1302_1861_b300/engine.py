"""Run a workload through the C ABI: upload, psl_build, psl_plan_create,
psl_source_batch + transport_run per piece of the history range, dose_readout.

PyTorch supplies device memory and streams; every computation is a call into
libpsl_b300.so.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import torch

from . import capi
from .inputs import Workload


@dataclasses.dataclass
class DeviceWorkload:
    """A workload's arrays on the GPU plus the C structs that point at them."""
    w: Workload
    rec_t: List[torch.Tensor]
    mat_t: torch.Tensor
    rho_t: torch.Tensor
    flu_t: List[Optional[torch.Tensor]]
    params: capi.Params
    records: capi.Records
    phantom: capi.Phantom
    beams: List[capi.Beam]
    _keep: list


def records_struct(ts: List[torch.Tensor]) -> capi.Records:
    r = capi.Records()
    r.x, r.y, r.u, r.v, r.e, r.wt, r.q = (t.data_ptr() for t in ts)
    r.n = int(ts[0].shape[0])
    return r


def upload(w: Workload, device: str = "cuda", records=None) -> DeviceWorkload:
    """Copy a workload to the device.  `records` may give tensors already there."""
    if records is None:
        rec_t = [torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in w.records.arrays()]
    else:
        rec_t = list(records)
    b = w.binning
    xe, ye, ee = (np.ascontiguousarray(a, np.float32) for a in (b.x_edges, b.y_edges, b.e_edges))
    params = capi.Params(b.nx, b.ny, b.n_ebins, int(b.apr_copies), xe.ctypes.data, ye.ctypes.data, ee.ctypes.data,
                         float(w.z_psl), int(b.apr_seed))
    ph = w.phantom
    nz, ny, nx = ph.shape
    mat_t = torch.from_numpy(np.ascontiguousarray(ph.mat, np.uint8)).to(device)
    rho_t = torch.from_numpy(np.ascontiguousarray(ph.rho, np.float32)).to(device)
    phantom = capi.Phantom(nx, ny, nz, *map(float, ph.voxel), (capi.f32 * 3)(*map(float, ph.origin)),
                           mat_t.data_ptr(), rho_t.data_ptr())
    beams, flu_t = [], []
    for bm in w.beams:
        f = None if bm.fluence is None else torch.from_numpy(np.ascontiguousarray(bm.fluence, np.float32)).to(device)
        flu_t.append(f)
        fny, fnx = (0, 0) if f is None else f.shape
        beams.append(capi.Beam(bm.x1, bm.x2, bm.y1, bm.y2, bm.z_jaw_x, bm.z_jaw_y, bm.gantry, bm.collimator,
                               bm.couch, bm.mu, bm.roi_margin, (capi.f32 * 3)(*map(float, bm.iso)), fnx, fny,
                               bm.fx0, bm.fy0, bm.fdx, bm.fdy, 0 if f is None else f.data_ptr()))
    return DeviceWorkload(w, rec_t, mat_t, rho_t, flu_t, params, records_struct(rec_t), phantom, beams,
                          [xe, ye, ee])


def shard_histories(rank: int, world: int, per_rank: int):
    """Weak scaling over ranks: rank r transports histories [r N, (r+1) N) of
    a plan of world * N histories.  Histories are independent, their random
    streams are keyed by history id and the tally is an integer sum, so the
    shards' tallies add up to the unsharded one exactly."""
    return rank * per_rank, per_rank, world * per_rank


def chunks(first: int, n: int, size: int):
    """Contiguous pieces [f, f + c) of the history range [first, first+n)."""
    size = max(1, int(size))
    return [(f, min(size, first + n - f)) for f in range(first, first + n, size)]


def normalisation(plan, n_histories: int, n_incident: int = 0, calibration: float = 1.0) -> float:
    """Sec. 2.5 normalisation, computed by the library (psl_dose_normalisation):
    N_total^psl / (N_simulated N_incident) x calibration.  n_incident = 0 takes
    the store's records x redistribution copies (a synthetic phase space is
    its own incident set)."""
    return capi.dose_normalisation(plan, n_histories, n_incident, calibration)


class _DeviceInt64:
    """A library-owned device int64 array seen by torch without a copy."""

    def __init__(self, addr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i8", "data": (int(addr), False),
                                         "version": 3, "strides": None}


def tally_views(tally):
    """Torch views (no copy) of a tally's int64 counters [n_batches * nvox]
    and its 12-slot ledger, on the current CUDA device."""
    n, _, _, _ = capi.psl_tally_info(tally)
    t_addr, l_addr = capi.psl_tally_buffers(tally)
    t = torch.as_tensor(_DeviceInt64(t_addr, n), device="cuda")
    lg = torch.as_tensor(_DeviceInt64(l_addr, 12), device="cuda")
    return t, lg


def sum_over_ranks(counters, ledger, group=None) -> None:
    """Element-wise int64 SUM of a tally's counters and ledger over the
    ranks of `group`, in place (torch.distributed): device tensors on NCCL
    directly, otherwise through host copies (gloo); host tensors directly."""
    import torch.distributed as dist
    if counters.is_cuda and dist.get_backend(group) != "nccl":
        th, lh = counters.cpu(), ledger.cpu()
        dist.all_reduce(th, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(lh, op=dist.ReduceOp.SUM, group=group)
        counters.copy_(th)
        ledger.copy_(lh)
        return
    dist.all_reduce(counters, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(ledger, op=dist.ReduceOp.SUM, group=group)


def reduce_tallies(tally, group=None) -> None:
    """Sec. 2.3.3 (a job split over GPUs): sum every rank's tally and ledger
    into every rank's, in place, on the tally's own device arrays.  Each
    history runs on one rank and the counters are integers, so the sum is
    the tally of the whole range bit for bit; dose_readout follows on it.
    Call it after the rank's transport calls (psl_run and transport_run
    synchronise their stream before returning)."""
    t, lg = tally_views(tally)
    sum_over_ranks(t, lg, group)


def run(dw: DeviceWorkload, n_histories: Optional[int] = None, n_batches: Optional[int] = None,
        flags: int = 0, store=None, plan=None, tally=None, readout: bool = True, stream=None,
        batch_size: int = 1 << 24):
    """Whole plan on the GPU.  Returns a dict with the handles and (device) dose."""
    w = dw.w
    n_sim = w.n_histories
    n_h = n_sim if n_histories is None else n_histories
    nb = w.n_batches if n_batches is None else n_batches
    if store is None:
        store = capi.psl_build(dw.params, dw.records, stream)
    if plan is None:
        plan = capi.psl_plan_create(store, dw.beams, w.sad, n_sim, w.seed, stream)
    if tally is None:
        tally = capi.psl_tally_create(dw.phantom, nb)
    phys = capi.physics(flags)
    # histories in reading order, one psl_source_batch per piece; every
    # history's deposits go to the tally slice (batch) of its id
    for f0, cnt in chunks(0, n_h, batch_size):
        batch = capi.psl_source_batch(plan, dw.phantom, f0, cnt, 1, stream)
        capi.transport_run(dw.phantom, phys, batch, tally, capi.SLICE_BY_HISTORY, stream)
        batch.close()
    out = dict(store=store, plan=plan, tally=tally)
    if readout:
        nvox = dw.mat_t.numel()
        dose = torch.empty(nvox, dtype=torch.float64, device=dw.mat_t.device)
        sigma = torch.empty_like(dose)
        ledger = torch.empty(3, dtype=torch.float64, device=dose.device)
        norm = normalisation(plan, n_h)
        capi.dose_readout(tally, dw.phantom, norm, dose, sigma, ledger, stream)
        out.update(dose=dose, sigma=sigma, ledger=ledger, norm=norm)
    return out


def raw_tallies(dw: DeviceWorkload, tally, n_batches: int):
    nz, ny, nx = dw.w.phantom.shape
    t = torch.empty(n_batches * nz * ny * nx, dtype=torch.int64, device=dw.mat_t.device)
    lg = torch.empty(12, dtype=torch.int64, device=t.device)
    capi.psl_tally_read(tally, t, lg)
    torch.cuda.synchronize()
    return t.view(n_batches, nz, ny, nx).cpu().numpy(), lg.cpu().numpy()
