"""The dose denoiser around the PSL Monte Carlo: training pairs generated by
the method itself, training, inference and its accuracy check.

A pair is (low-history dose, density) -> high-history dose on the same
geometry; the low-history doses are independent runs (their own plan seeds).
Every dose comes from psl_build / psl_plan_create / psl_run / dose_readout,
every network step from psl_denoiser_*; this module only sequences the calls
and cuts 64^3 crops.  Accuracy is judged against a plain high-history run by
the gamma index (psl_gamma), and the plain run to 1 % uncertainty is the
fallback the denoised result has to beat in time.

    python -m paper_1302_1861_b300.denoiser --out weights.npy
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time
from typing import List, Optional

import numpy as np
import torch

from . import capi, engine, inputs

CROP = 64
# Dose is estimated in the body only: voxels below this density (the air
# around a CT body, 0.001 g/cm^3) hold doses of a few deposits in a tiny mass
# that would dominate the loss and the dose maximum, so the network's input
# and target are zero there and the accuracy is judged on the body.
BODY_RHO = 0.1


@dataclasses.dataclass
class Pair:
    lo: torch.Tensor          # float32 [z, y, x] low-history dose (device)
    rho: torch.Tensor         # float32 density
    hi: torch.Tensor          # float32 high-history dose
    scale: float


def body(dose: torch.Tensor, rho: torch.Tensor) -> torch.Tensor:
    """The dose with the voxels outside the body (rho < BODY_RHO) set to 0."""
    return torch.where(rho.view(dose.shape) >= BODY_RHO, dose, torch.zeros_like(dose))


def dose_scale(dose: torch.Tensor) -> float:
    """Normalisation of a dose for the network: its 99.9th percentile, the
    k-th smallest value with k = max(1, floor(0.999 n)) counted from 1
    (robust against single noisy voxels), found on the device."""
    flat = dose.reshape(-1).float().contiguous()
    k = max(1, int(0.999 * flat.numel()))
    v = capi.kth_smallest(flat, k - 1)
    return v if v > 0 else 1.0


class DoseRunner:
    """Plain PSL Monte Carlo doses on one phase space, for any phantom and
    field list (a store built once, a plan and a tally per call)."""

    def __init__(self, w: inputs.Workload):
        self.w = w
        self.dw = engine.upload(w)
        self.store = capi.psl_build(self.dw.params, self.dw.records)
        self.phys = capi.physics()

    def geometry(self, phantom: inputs.Phantom, beams) -> engine.DeviceWorkload:
        w2 = dataclasses.replace(self.w, phantom=phantom, beams=beams)
        return engine.upload(w2, records=self.dw.rec_t)

    def dose(self, g: engine.DeviceWorkload, n: int, seed: int, n_batches: int = 10):
        """(dose, sigma) float64 [nz, ny, nx] on the device, and seconds."""
        w = g.w
        nz, ny, nx = w.phantom.shape
        tally = capi.psl_tally_create(g.phantom, n_batches)
        dose = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
        sigma = torch.empty_like(dose)
        lg = torch.empty(3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = capi.psl_plan_create(self.store, g.beams, w.sad, n, seed)
        capi.psl_run(plan, g.phantom, self.phys, tally, 0, n)
        _, n_total, _ = plan.info()
        capi.dose_readout(tally, g.phantom, engine.normalisation(plan, n),
                          dose, sigma, lg)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        plan.close()
        tally.close()
        return dose.view(nz, ny, nx), sigma.view(nz, ny, nx), secs


def _crops(shape, rng, count):
    """Corners of `count` random CROP^3 crops aligned to 8 voxels."""
    out = []
    for _ in range(count):
        out.append(tuple(int(rng.integers(0, (s - CROP) // 8 + 1)) * 8 for s in shape))
    return out


def make_pairs(n_slab: int = 16, n_ct: int = 16, lo_per_geometry: int = 10, n_hi: int = 2_000_000_000,
               n_lo=(1_000_000, 10_000_000), n_hi_ct: int = 4_000_000_000, n_lo_ct=(30_000_000, 300_000_000),
               lo_per_ct: int = 8, crops_per_ct: int = 4, seed: int = 7, log=print) -> List[Pair]:
    """Training pairs from seeded slab (64^3, whole volume) and CT (128^3,
    64^3 crops) geometries: one high-history target per geometry and
    independent low-history runs with log-uniform history counts (n_lo for
    the slabs, n_lo_ct for the CT volumes, whose 8x more voxels need more
    histories for the same noise).  Doses outside the body are zeroed."""
    rng = np.random.default_rng(seed)
    pairs: List[Pair] = []
    for kind, count, base, nh, nl, per in (("slab", n_slab, inputs.config2(n_histories=1000), n_hi, n_lo, lo_per_geometry),
                                           ("ct", n_ct, inputs.config3(n_histories=1000), n_hi_ct, n_lo_ct, lo_per_ct)):
        if count == 0:
            continue
        runner = DoseRunner(base)
        for g in range(count):
            phantom, beams = inputs.denoiser_geometry(kind, g)
            geo = runner.geometry(phantom, beams)
            rho = torch.from_numpy(np.ascontiguousarray(phantom.rho, np.float32)).cuda()
            hi, _, t_hi = runner.dose(geo, nh, 10_000 + g)
            hi = body(hi, rho)
            for r in range(per):
                n = int(np.exp(rng.uniform(np.log(nl[0]), np.log(nl[1]))))
                lo, _, _ = runner.dose(geo, n, 20_000 + 100 * g + r)
                lo = body(lo, rho)
                corners = [(0, 0, 0)] if kind == "slab" else _crops(phantom.shape, rng, crops_per_ct)
                for (z, y, x) in corners:
                    sl = (slice(z, z + CROP), slice(y, y + CROP), slice(x, x + CROP))
                    lo_c = lo[sl].float().contiguous()
                    pairs.append(Pair(lo_c, rho[sl].contiguous(), hi[sl].float().contiguous(), dose_scale(lo_c)))
            if log:
                log(f"{kind} geometry {g}: target {nh:.1e} histories in {t_hi:.2f} s, pairs {len(pairs)}")
    return pairs


class TrainingStalled(RuntimeError):
    """The loss stopped falling in the first epochs: the ReLUs of the
    decoder died and the network is stuck at the identity on the dose."""


def train(den: capi.Denoiser, pairs: List[Pair], epochs: int = 30, lr: float = 2e-3, batch: int = 4, seed: int = 0,
          log=print, stall_epoch: int = 3) -> List[float]:
    """Adam on the mean squared error (in units of each pair's scale), a
    cosine learning-rate decay to lr / 20; returns the mean loss per epoch.
    Raises TrainingStalled when the loss of epoch `stall_epoch` is above 0.9
    of the first epoch's (healthy runs fall ~7x by epoch 5; a run on 24 CT
    geometries stayed at the identity from its first epoch)."""
    rng = np.random.default_rng(seed)
    hist = []
    steps = epochs * ((len(pairs) + batch - 1) // batch)
    k = 0
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for i in range(0, len(order), batch):
            for j in order[i:i + batch]:
                p = pairs[j]
                nz, ny, nx = p.lo.shape
                tot += den.backward(p.lo, p.rho, p.hi, nx, ny, nz, p.scale)
            lr_k = lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * k / max(steps, 1))))
            den.step(float(lr_k))
            k += 1
        hist.append(tot / len(pairs))
        if log and (ep % 5 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {hist[-1]:.3e}")
        if ep == stall_epoch and hist[-1] > 0.9 * hist[0]:
            raise TrainingStalled(f"loss {hist[0]:.3e} -> {hist[-1]:.3e} after {ep} epochs")
    return hist


def denoise(den: capi.Denoiser, dose: torch.Tensor, rho: torch.Tensor, scale: Optional[float] = None) -> torch.Tensor:
    """The denoised dose (float32, device) of a dose volume whose sides are
    multiples of 8 (estimated in the body; 0 input outside it)."""
    nz, ny, nx = dose.shape
    d32 = body(dose.float(), rho).contiguous()
    out = torch.empty_like(d32)
    den.forward(d32, rho.float().contiguous(), nx, ny, nz, scale or dose_scale(d32), out)
    return out


def save(den: capi.Denoiser, path: str):
    p = torch.empty(capi.Denoiser.param_count(), dtype=torch.float32, device="cuda")
    den.params(get=p)
    np.save(path, p.cpu().numpy())


def load(path: str) -> capi.Denoiser:
    den = capi.Denoiser.create(0)
    p = torch.from_numpy(np.load(path).astype(np.float32)).cuda()
    den.params(set=p)
    return den


def errors(ref: torch.Tensor, ev: torch.Tensor, voxel, rho: Optional[torch.Tensor] = None) -> dict:
    """Accuracy of ev against ref in the body (both zeroed where rho <
    BODY_RHO, when rho is given): gamma pass rates (2 %/2 mm and 1 %/1 mm,
    voxels above 10 % of the maximum) and the RMS relative dose error over the
    voxels above 50 % of the maximum (gamma alone flatters noisy doses: the
    search finds a matching value next to most noisy voxels)."""
    if rho is not None:
        ref, ev = body(ref, rho).contiguous(), body(ev, rho).contiguous()
    g2, n_eval = capi.gamma(ref, ev, voxel)
    g1, _ = capi.gamma(ref, ev, voxel, dose_crit=0.01, dta_cm=0.1)
    m = ref > 0.5 * ref.max()
    rms = float(torch.sqrt((((ev[m] - ref[m]) / ref[m]) ** 2).mean()))
    return {"gamma_2pct_2mm": g2, "gamma_1pct_1mm": g1, "rms_rel_error_50pct": rms, "voxels": n_eval}


def evaluate(den: capi.Denoiser, runner: DoseRunner, geo: engine.DeviceWorkload, n_lo: int, ref: torch.Tensor,
             seed: int = 99):
    """A low-history run, denoised, against a reference dose: accuracy of the
    noisy and the denoised dose, the seconds of MC + inference, and the plain
    histories that would give the denoised RMS error (RMS error of plain runs
    falls as 1/sqrt(N))."""
    w = geo.w
    lo, _, t_mc = runner.dose(geo, n_lo, seed)
    rho = torch.from_numpy(np.ascontiguousarray(w.phantom.rho, np.float32)).cuda()
    denoise(den, lo, rho)                      # first call on this shape sets up its buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dn = denoise(den, lo, rho)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    e_lo = errors(ref, lo, w.phantom.voxel, rho)
    e_dn = errors(ref, dn.double().contiguous(), w.phantom.voxel, rho)
    eq = n_lo * (e_lo["rms_rel_error_50pct"] / max(e_dn["rms_rel_error_50pct"], 1e-12)) ** 2
    return {"histories": n_lo, "noisy": e_lo, "denoised": e_dn, "equivalent_plain_histories": eq,
            "mc_seconds": t_mc, "inference_seconds": t_inf, "seconds": t_mc + t_inf}


def held_out_report(den: capi.Denoiser, n_ref=(4_000_000_000, 4_000_000_000),
                    n_lo=((3_000_000, 10_000_000), (30_000_000, 100_000_000, 300_000_000)), log=print,
                    plain_1pct=None) -> dict:
    """Accuracy and time of the denoised form on geometries not trained on:
    the 10x10 field on its slab phantom and the 30x30 fluence field on its
    CT-like phantom, each against a plain high-history reference.
    plain_1pct: optional {workload name: measured plain run to 1 %} that
    replaces the extrapolation from the reference."""
    rep = {}
    for (name, w), nr, nl in zip((("psl-10x10-slab64", inputs.config2(n_histories=1000)),
                                  ("psl-30x30-ct128", inputs.config3(n_histories=1000))), n_ref, n_lo):
        runner = DoseRunner(w)
        ref, sig, t_ref = runner.dose(runner.dw, nr, 4242)
        # the plain run to 1 % isocentre uncertainty (mean sigma/D over the
        # 3x3x3 isocentre voxels), extrapolated from the reference as 1/sqrt(N)
        c = ((np.array(w.beams[0].iso) - np.array(w.phantom.origin)) / np.array(w.phantom.voxel)).astype(int)[::-1]
        sl = tuple(slice(k - 1, k + 2) for k in c)
        rel = float((sig[sl] / ref[sl]).mean())
        n1 = nr * (rel / 0.01) ** 2
        p1 = {"histories": n1, "seconds": t_ref * n1 / nr, "kind": "extrapolated from the reference"}
        if plain_1pct and plain_1pct.get(name):
            p1 = plain_1pct[name]
        rep[name] = {"reference_histories": nr, "reference_seconds": t_ref, "plain_to_1pct": p1,
                     "runs": [evaluate(den, runner, runner.dw, n, ref, seed=77 + i) for i, n in enumerate(nl)]}
        if log:
            log(f"{name}: {rep[name]}")
    return rep


def main():
    ap = argparse.ArgumentParser(description="train the dose denoiser on pairs generated by the PSL method")
    ap.add_argument("--out")
    ap.add_argument("--report", default=None, help="write the held-out accuracy report (JSON) here")
    ap.add_argument("--slab", type=int, default=16)
    ap.add_argument("--ct", type=int, default=16)
    ap.add_argument("--lo-per-geometry", type=int, default=10)
    ap.add_argument("--n-hi", type=float, default=2e9)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args()
    if not a.out:
        ap.error("--out is required for training")
    t0 = time.perf_counter()
    pairs = make_pairs(a.slab, a.ct, a.lo_per_geometry, int(a.n_hi))
    t1 = time.perf_counter()
    # a stalled start (dead ReLUs) is restarted from the next seed's weights
    for attempt in range(3):
        den = capi.Denoiser.create(a.seed + attempt)
        try:
            hist = train(den, pairs, a.epochs, a.lr)
            break
        except TrainingStalled as e:
            print(f"seed {a.seed + attempt}: {e}; restarting from seed {a.seed + attempt + 1}", flush=True)
            den.close()
    else:
        raise SystemExit("training stalled from three initial weight sets")
    t2 = time.perf_counter()
    save(den, a.out)
    summary = {"pairs": len(pairs), "pair_seconds": t1 - t0, "train_seconds": t2 - t1, "loss": hist}
    print(json.dumps({k: v for k, v in summary.items() if k != "loss"}), flush=True)
    if a.report:
        summary["held_out"] = held_out_report(den)
        with open(a.report, "w") as f:
            json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
