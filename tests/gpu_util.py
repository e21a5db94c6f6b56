"""Helpers shared by the GPU parity tests (not a test module)."""
import numpy as np
import torch

from paper_1302_1861_b300 import capi, engine


def store_arrays(store, n_bins, n_valid):
    off = torch.empty(n_bins + 1, dtype=torch.int64, device="cuda")
    perm = torch.empty(max(n_valid, 1), dtype=torch.int64, device="cuda")
    rec = torch.empty(max(n_valid, 1) * 8, dtype=torch.float32, device="cuda")
    capi.psl_store_read(store, off, perm, rec)
    torch.cuda.synchronize()
    return off.cpu().numpy(), perm.cpu().numpy()[:n_valid], rec.cpu().numpy()[: n_valid * 8].reshape(-1, 8)


def plan_arrays(plan):
    n_entries, n_total, n_hist = plan.info()
    a = [torch.empty(n_entries, dtype=torch.int64, device="cuda") for _ in range(4)]
    capi.psl_plan_read(plan, *a)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in a], n_total


def source_trace(dw, plan, h0, n, stride=1):
    d = dict(entry=torch.empty(n, dtype=torch.int64, device="cuda"),
             use=torch.empty(n, dtype=torch.int64, device="cuda"),
             rec=torch.empty(n, dtype=torch.int64, device="cuda"),
             beam=torch.empty(n, dtype=torch.int32, device="cuda"),
             status=torch.empty(n, dtype=torch.int8, device="cuda"),
             state=torch.empty(n * 8, dtype=torch.float32, device="cuda"),
             ptype=torch.empty(n, dtype=torch.int32, device="cuda"))
    capi.psl_source_trace(plan, dw.phantom, h0, n, stride=stride, **d)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in d.items()}
    out["state"] = out["state"].reshape(n, 8)
    return out


def transport_particles(dw, ptype, pos, dirs, e, wt, pid, seed, flags=0, trace=False):
    """Transport caller particles (phantom-local) on the GPU; returns the
    int64 tally, ledger and (optionally) per-particle sums."""
    n = len(e)
    state = np.concatenate([np.asarray(pos, np.float32), np.asarray(dirs, np.float32),
                            np.asarray(e, np.float32)[:, None], np.asarray(wt, np.float32)[:, None]], 1)
    st = torch.from_numpy(np.ascontiguousarray(state)).cuda()
    pt = torch.from_numpy(np.ascontiguousarray(ptype, np.int32)).cuda()
    pd = torch.from_numpy(np.ascontiguousarray(pid, np.uint64).view(np.int64)).cuda()
    batch = capi.psl_batch_from_particles(st, pt, pd, seed)
    tally = capi.psl_tally_create(dw.phantom, 1)
    hd = he = hv = None
    if trace:
        hd = torch.zeros(n, dtype=torch.int64, device="cuda")
        he = torch.zeros(n, dtype=torch.int64, device="cuda")
        hv = torch.zeros(n, dtype=torch.int32, device="cuda")
    capi.transport_trace(dw.phantom, capi.physics(flags), batch, tally, 0, hd, he, hv)
    t, lg = engine.raw_tallies(dw, tally, 1)
    tally.close()
    batch.close()
    if trace:
        return t[0], lg, dict(dep=hd.cpu().numpy(), esc=he.cpu().numpy(), events=hv.cpu().numpy())
    return t[0], lg
