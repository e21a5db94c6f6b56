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


def normalisation(n_total_psl: int, n_histories: int, n_incident: int) -> float:
    """Sec. 2.5: D = D_o N^phsp / (N_simulated N_incident); with PSL selection the
    histories stand for the N_total^psl selected records.  With azimuthal
    redistribution a phase space of N records and K copies stands for K N
    incident particles (pass n_incident = K N)."""
    return float(n_total_psl) / (float(n_histories) * float(n_incident))


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
        _, n_total_psl, _ = plan.info()
        norm = normalisation(n_total_psl, n_h, w.records.n * int(w.binning.apr_copies))
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
