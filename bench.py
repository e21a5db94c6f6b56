#!/usr/bin/env python
"""Benchmark of the PSL Monte Carlo dose path on one B300 (or N, one rank per GPU).

Headline workload (the 30x30 cm^2 configuration, the largest that runs on
one GPU): a patient-independent phase space of 4e7 records over 40 x 40 cm
(2 types x 32 log-energy x 40 x 40 1-cm PSL bins = 102,400 PSLs), 30x30 cm
jaws with a 40x40 fluence map, a 128^3 x 0.25 cm CT-like phantom, 1e9
histories in 10 batches.  One step is the whole path on that input:
psl_build (sort the phase space into PSLs), psl_plan_create, psl_run over
the rank's histories (each history's deposits into its batch), with N > 1
ranks the int64 sum of every rank's tally, and dose_readout.  The metric is
histories per second (whole job, all ranks); the inputs (1 GB of records)
are resident in HBM and larger than L2, and L2 is also flushed between
steps.

Extra keys: `e2e` (the same step through the C ABI from pinned host buffers,
with the records/phantom uploaded and dose/sigma/ledger read back inside the
timed region), `modes` (the plain form, psl_source_batch + transport_run
batch by batch), `roofline` (dominant kernel, timed live with CUDA events on
its stream), `cpu_baseline` (the oracle on a bounded stratified sample on
the host cores), `time_to_1pct` (a whole plan timed from psl_build to
dose_readout, its histories raised until the isocentre uncertainty is
<= 1 %), `workload_10x10` (the 10x10 slab workload: histories/s and its
measured time to 1 %), `imrt_batched_graph` (the IMRT plan autotuned and in
one CUDA-graph launch, and its time to 1 % measured the same way),
`methods`, `apr_build`, `denoised`, `transport`, `tally_memory`, `clocks`,
`gpu_launches`.

`--impl reference` times the CPU oracle as the reference arm, on the same
workload and the same sample size.  `--conv N CI CO` only times the
denoiser's convolution kernel (for profiling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "histories/s (PSL source + transport + dose readout)"
PEAKS_FALLBACK = {"hbm_gbs": 6400.0}
# FP32 CUDA-core peak: 148 SMs x 128 lanes x 2 flop x 2.032 GHz
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML
    polled every 10 ms from a thread (the device found by its UUID), else
    nvidia-smi at its 200 ms interval.  Read-only queries; nothing is set."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []          # (sm MHz, max sm MHz, reason names)
        self.nvml_error = None
        self.done = threading.Event()

    def _nvml_handle(self):
        """NVML (read-only queries, through ctypes on the driver's
        libnvidia-ml) and the handle of CUDA device `index`: by its UUID,
        else the only device NVML sees."""
        import ctypes
        import torch
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        u = str(getattr(torch.cuda.get_device_properties(self.index), "uuid", ""))
        for cand in ([u, "GPU-" + u] if u else []):
            if lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(cand.encode()), ctypes.byref(h)) == 0:
                return lib, h
        n = ctypes.c_uint()
        if lib.nvmlDeviceGetCount_v2(ctypes.byref(n)) == 0 and n.value == 1 and \
                lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(0), ctypes.byref(h)) == 0:
            return lib, h
        raise RuntimeError(f"no NVML device for CUDA device {self.index} (uuid {u})")

    def start(self):
        try:
            import ctypes
            lib, h = self._nvml_handle()
            NVML_CLOCK_SM = 1
            # clock event reason bits of nvml.h: sw power cap 0x4, hw slowdown
            # 0x8, sw thermal 0x20, hw thermal 0x40
            bits = [0x8, 0x40, 0x20, 0x4]
            v = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(v)) != 0:
                raise RuntimeError("nvmlDeviceGetMaxClockInfo failed")
            smax = float(v.value)
            self.nvml = lib

            def poll():
                c, r = ctypes.c_uint(), ctypes.c_ulonglong()
                while not self.done.is_set():
                    if lib.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(c)) == 0 and \
                            lib.nvmlDeviceGetCurrentClocksThrottleReasons(h, ctypes.byref(r)) == 0:
                        self.samples.append((float(c.value), smax,
                                             [n for n, b in zip(self.NAMES, bits) if r.value & b]))
                    self.done.wait(0.01)
            self.th = threading.Thread(target=poll, daemon=True)
            self.th.start()
            return
        except Exception as e:            # noqa: BLE001 - fall back to nvidia-smi
            self.nvml = None
            self.nvml_error = str(e)[:200]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.done.set()
            self.th.join(timeout=5)
            self.nvml.nvmlShutdown()
            src = "nvml, 10 ms"
        elif self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            for ln in self.lines:
                f = [x.strip() for x in ln.split(",")]
                if len(f) < 9:
                    continue
                try:
                    self.samples.append((float(f[1]), float(f[2]),
                                         [n for n, v in zip(self.NAMES, f[5:9]) if v.lower() == "active"]))
                except ValueError:
                    continue
            src = "nvidia-smi, 200 ms"
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "nvml_error": self.nvml_error}
        sm = [x[0] for x in self.samples]
        smax = [x[1] for x in self.samples]
        reasons = sorted({n for x in self.samples for n in x[2]})
        out = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "sm_min_mhz": min(sm) if sm else None, "reasons": reasons, "samples": len(sm), "source": src}
        if self.nvml_error:
            out["nvml_error"] = self.nvml_error
        return out


# --------------------------------------------------------------------------
def oracle_setup(w):
    """The oracle's PSL build and plan of the whole phase space (timed)."""
    from oracle import source
    t0 = time.perf_counter()
    st = source.psl_build(w.records, w.binning)
    pl = source.make_plan(st, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)
    return st, pl, time.perf_counter() - t0


def oracle_sample_seconds(w, st, pl, n_sample, nthreads, offset=0):
    """Seconds the oracle takes for `n_sample` histories of the plan: 20
    runs of n_sample / 20 consecutive histories, one in each twentieth of
    the reading order (it is energy major, so every stratum is sampled),
    shifted by `offset` within its stratum; source stage and transport."""
    import oracle
    from oracle import source
    k = 20
    per = max(1, n_sample // k)
    stride = w.n_histories // k
    tot = 0.0
    for j in range(k):
        h0 = j * stride + (offset % max(1, stride - per))
        hs = np.arange(h0, h0 + per)
        t = time.perf_counter()
        s = source.source(pl, st, w.records, w.beams, w.phantom, hs, w.z_psl, w.sad)
        m = s.status == source.ST_TRANSPORT
        oracle.transport(s.ptype[m], s.pos[m], s.dir[m], s.e[m], s.wt[m].astype(float),
                         hs[m].astype(np.uint64), w.phantom, w.seed, nthreads=nthreads)
        tot += time.perf_counter() - t
    return tot, per * k


def headline_workload():
    from paper_1302_1861_b300 import inputs
    return inputs.config3()


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm, on the headline workload: the
    oracle's PSL build and plan of all records once, then each step a
    bounded stratified sample of the plan's histories on every host core,
    the whole-plan time scaled from the setup and the per-history time."""
    if rank != 0:
        return
    w = headline_workload()
    st, pl, t_setup = oracle_setup(w)
    n_s = args.ref_sample
    rng = np.random.default_rng(7)
    # every host core (a launcher's OMP_NUM_THREADS=1 is meant for the GPU ranks)
    cores = os.cpu_count()

    def step():
        secs, n = oracle_sample_seconds(w, st, pl, n_s, cores, int(rng.integers(0, 1 << 30)))
        return secs / n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    t_h = float(np.mean([step() for _ in range(args.steps)]))
    t_sample = (time.perf_counter() - t0) / max(args.steps, 1)
    value = w.n_histories / (t_setup + t_h * w.n_histories)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * (t_setup + t_h * w.n_histories), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, w.n_histories, world),
            "cpu_baseline": {"value": value, "unit": "histories/s", "cores": cores, "kind": "oracle",
                             "sample": f"psl_build+plan of all {w.records.n} records ({t_setup:.2f} s) + per step "
                                       f"{n_s} histories in 20 strata of the reading order "
                                       f"({t_h * n_s:.2f} s), scaled to {w.n_histories} histories"},
            "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_ms_per_step": 1e3 * t_sample,
            "note": "ms_per_step is the whole 1e9-history step extrapolated from the oracle's setup time and the "
                    "per-history time of each step's sample; sample_ms_per_step is the wall time a step's sample "
                    "took"}
    print(json.dumps(line))


def cpu_baseline(w, n_sample):
    """The oracle as it stands on a bounded sample of the headline workload:
    the same setup and the same stratified sample size as the reference arm,
    on every host core, and a quarter of it on one thread."""
    st, pl, t_setup = oracle_setup(w)
    cores = os.cpu_count()
    secs, n = oracle_sample_seconds(w, st, pl, n_sample, cores)
    t_h = secs / n
    value = w.n_histories / (t_setup + t_h * w.n_histories)
    secs1, n1 = oracle_sample_seconds(w, st, pl, n_sample // 4, 1)
    t_h1 = secs1 / n1
    return {"value": value, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"psl_build+plan of all {w.records.n} records ({t_setup:.2f} s) + {n} histories in 20 strata "
                      f"of the reading order ({secs:.2f} s), scaled to {w.n_histories} histories",
            "one_thread": {"value": w.n_histories / (t_setup + t_h1 * w.n_histories), "unit": "histories/s",
                           "sample": f"the same setup + {n1} histories on 1 thread ({secs1:.2f} s)"}}


def workload_config(w, per_rank, world):
    phantoms = {"psl-10x10-slab64": "64^3 x 0.25 cm water + lung/bone slabs",
                "psl-30x30-ct128": "128^3 x 0.25 cm CT-like (air, lung, soft tissue, bone ellipsoids)"}
    return {"workload": w.name, "records": w.records.n, "psl_bins": w.binning.n_bins,
            "field": "30x30 cm jaws + 40x40 fluence map" if w.index == 3 else "10x10 cm jaws",
            "phantom": phantoms.get(w.name, str(w.phantom.shape)), "histories_per_gpu": per_rank,
            "batches": w.n_batches, "l2": "inputs > L2 and L2 flushed between steps",
            "parallelism": f"history-range shards x{world}"}


class Ctx:
    """What the measurement helpers share: the torch / library modules, the
    run's ranks and the L2 flush buffer."""

    def __init__(self, torch, dist, capi, engine, inputs, rank, world, local, args):
        self.torch, self.dist, self.capi, self.engine, self.inputs = torch, dist, capi, engine, inputs
        self.rank, self.world, self.local, self.args = rank, world, local, args
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()
        self.torch.cuda.synchronize()

    def max_over_ranks(self, v):
        if self.world > 1:
            tt = self.torch.tensor([v], device="cuda", dtype=self.torch.float64)
            self.dist.all_reduce(tt, op=self.dist.ReduceOp.MAX)
            v = float(tt.item())
        return v


def make_step(c, w, tally, first, per_rank, n_plan):
    """psl_build + psl_plan_create + the rank's histories + (N > 1: the
    int64 sum of every rank's tally) + dose_readout.  Default: the rank's
    whole range in one psl_run call; plain: psl_source_batch +
    transport_run piece by piece (N_b pieces).  Every history's deposits go
    to the tally slice (batch) of its id."""
    capi, engine = c.capi, c.engine
    phys = capi.physics()

    def step(dwx, out, plain=False):
        store = capi.psl_build(dwx.params, dwx.records)
        plan = capi.psl_plan_create(store, dwx.beams, w.sad, n_plan, w.seed)
        capi.psl_tally_reset(tally)
        if plain:
            for f0, cnt in engine.chunks(first, per_rank, -(-per_rank // w.n_batches)):
                batch = capi.psl_source_batch(plan, dwx.phantom, f0, cnt, 1)
                capi.transport_run(dwx.phantom, phys, batch, tally, capi.SLICE_BY_HISTORY)
                batch.close()
        else:
            capi.psl_run(plan, dwx.phantom, phys, tally, first, per_rank)
        if c.world > 1:
            engine.reduce_tallies(tally)                # one dose from all ranks' histories
        norm = engine.normalisation(plan, per_rank * c.world)
        capi.dose_readout(tally, dwx.phantom, norm, out[0], out[1], out[2])
        return store, plan
    return step


def timed_steps(c, step, dw, out, steps, plain=False):
    """Device time of `steps` steps (CUDA events on the launching stream,
    barrier + synchronize on both sides, L2 flushed before each)."""
    torch = c.torch
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        c.flush.fill_(1.0)
        c.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(dw, out, plain)
        e1.record(stream)
        c.barrier()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times


def isocentre_slice(w):
    iso = np.array(w.beams[0].iso) - np.array(w.phantom.origin)
    ic = (iso / np.array(w.phantom.voxel)).astype(int)[::-1]
    return tuple(slice(k - 1, k + 2) for k in ic)


def e2e_run(c, w, step, out, steps, warmup):
    """End to end through the C ABI: every step uploads its records and
    phantom from pinned host memory and reads back dose, sigma and ledger,
    all inside the timed region.  Double-buffered: step k+1's inputs go up
    on a copy stream while step k computes (the copy engine runs beside the
    kernels), as a service taking plan after plan would stream them."""
    torch, engine = c.torch, c.engine
    stream = torch.cuda.current_stream()
    nvox = int(np.prod(w.phantom.shape))
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w.records.arrays()]
    host_mat = torch.from_numpy(np.ascontiguousarray(w.phantom.mat)).pin_memory()
    host_rho = torch.from_numpy(np.ascontiguousarray(w.phantom.rho)).pin_memory()
    dws = [engine.upload(w, records=[torch.empty_like(h, device="cuda") for h in host]) for _ in range(2)]
    out_h = torch.empty(2 * nvox + 3, dtype=torch.float64).pin_memory()
    bi = sum(h.numel() * h.element_size() for h in host) + host_mat.numel() + host_rho.numel() * 4
    bo = out_h.numel() * 8
    cstream = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    for e in ev_free:
        e.record(stream)

    def upload(slot):
        with torch.cuda.stream(cstream):
            cstream.wait_event(ev_free[slot])            # the step that used this buffer is done
            for hh, dd in zip(host, dws[slot].rec_t):
                dd.copy_(hh, non_blocking=True)
            dws[slot].mat_t.copy_(host_mat, non_blocking=True)
            dws[slot].rho_t.copy_(host_rho, non_blocking=True)
            ev_in[slot].record(cstream)

    def run(k_steps):
        upload(0)
        for k in range(k_steps):
            slot = k & 1
            if k + 1 < k_steps:
                upload(slot ^ 1)
            stream.wait_event(ev_in[slot])
            c.flush.fill_(1.0)
            step(dws[slot], out)
            ev_free[slot].record(stream)
            out_h[:nvox].copy_(out[0], non_blocking=True)
            out_h[nvox:2 * nvox].copy_(out[1], non_blocking=True)
            out_h[2 * nvox:].copy_(out[2], non_blocking=True)
        torch.cuda.synchronize()

    run(warmup)
    c.barrier()
    t0 = time.perf_counter()
    run(steps)
    te = c.max_over_ranks((time.perf_counter() - t0) / steps)
    del dws
    return te, int(bi), int(bo)


def measure(c, w, steps, warmup, with_e2e, with_t1pct, with_plain, profile=False):
    """The workload's step timed on this rank's history shard, and what
    goes with it: plain per-batch form, e2e, time to 1 %, counters."""
    torch, capi, engine = c.torch, c.capi, c.engine
    per_rank = w.n_histories if c.args.histories is None else c.args.histories
    # weak scaling: rank r transports histories [r*N, (r+1)*N) of a plan of world*N histories
    first, per_rank, n_plan = engine.shard_histories(c.rank, c.world, per_rank)
    dw = engine.upload(w)
    nz, ny, nx = w.phantom.shape
    nvox = nx * ny * nz
    out = (torch.empty(nvox, dtype=torch.float64, device="cuda"),
           torch.empty(nvox, dtype=torch.float64, device="cuda"),
           torch.empty(3, dtype=torch.float64, device="cuda"))
    tally = capi.psl_tally_create(dw.phantom, w.n_batches)       # device buffers held across steps
    capi.psl_tally_set_queue_depth(tally, c.args.queue_depth)
    step = make_step(c, w, tally, first, per_rank, n_plan)
    for _ in range(warmup):
        step(dw, out)
    c.barrier()
    clocks = ClockSampler(c.local) if profile else None
    if profile:
        capi.profile(True)
        n_launch0 = capi.kernel_launches()
        clocks.start()
    times = timed_steps(c, step, dw, out, steps)
    r = {"w": w, "per_rank": per_rank, "dw": dw, "tally": tally, "out": out}
    if profile:
        r["clocks"] = clocks.stop()
        r["launches"] = capi.kernel_launches() - n_launch0
        r["prof"] = capi.profile_read()
        capi.profile(False)
    t_step = c.max_over_ranks(float(np.mean(times)))
    r["t_step"] = t_step
    r["value"] = per_rank * c.world / t_step
    lg = out[2].cpu().numpy()
    raw = torch.empty(12, dtype=torch.int64, device="cuda")
    capi.psl_tally_read(tally, None, raw)
    r["counts"] = raw.cpu().numpy()            # event and atomic counters of the last step (all ranks)
    r["energy_balance"] = float((lg[1] + lg[2] - lg[0]) / lg[0])
    r["ledger_mev"] = [float(x) for x in lg]
    d = out[0].view(nz, ny, nx).cpu().numpy()
    s = out[1].view(nz, ny, nx).cpu().numpy()
    sl = isocentre_slice(w)
    rel = float((s[sl] / d[sl]).mean())
    r["iso_rel"] = rel
    n_1pct = per_rank * c.world * (rel / 0.01) ** 2
    if with_plain:
        pt = timed_steps(c, step, dw, out, 2, plain=True)
        r["plain"] = per_rank * c.world / c.max_over_ranks(float(np.mean(pt[1:])))
    if with_e2e:
        te, bi, bo = e2e_run(c, w, step, out, steps, warmup)
        r["e2e"] = {"value": per_rank * c.world / te, "unit": "histories/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo,
                    "note": "every step uploads its records and phantom from pinned host memory and reads back "
                            "dose, sigma and ledger; step k+1's upload runs on a copy stream during step k (two "
                            "device buffers); the first upload and the last read-back are inside the timed region"}
    # the step's tally (and its transport workspace) is released before the
    # whole-plan runs below take theirs
    r["tally_info"] = capi.psl_tally_info(tally)
    tally.close()
    del r["tally"]
    if with_t1pct and c.rank == 0 and c.world == 1:
        t1 = time_to_1pct(capi, torch, w, dw, capi.physics(), n_1pct, sl, (nz, ny, nx), c.args.queue_depth)
        t1["extrapolated_histories"] = n_1pct
        t1["extrapolated_seconds"] = n_1pct / (per_rank / t_step)
        r["t1pct"] = t1
    else:
        r["t1pct"] = {"histories": n_1pct, "seconds": n_1pct / r["value"], "isocentre_rel_sigma_at_run": rel,
                      "kind": "extrapolated from the run's sigma"}
    return r


def conv_only(args):
    """Only the tensor-core convolution of the denoiser on an n^3 volume,
    ci -> co channels (random BF16 data): two calls, then `steps` calls
    timed on the device with the library's events (for profiling one launch
    of its kernel)."""
    import torch
    from paper_1302_1861_b300 import capi
    n, ci, co = args.conv
    capi.conv3d_form(args.conv_form)
    x = torch.randn(n ** 3 * ci, device="cuda").to(torch.bfloat16)
    wt = torch.randn(27 * ci * co, device="cuda") * 0.05
    wpk = capi.conv3d_pack(wt, ci, co)
    out = torch.empty(n ** 3 * co, dtype=torch.bfloat16, device="cuda")
    for it in range(2):                                   # warm-up
        capi.conv3d(x.view(torch.int16), ci, wpk, None, co, n, n, n, True, out.view(torch.int16))
    capi.profile(True)
    for it in range(max(args.steps, 1)):
        capi.conv3d(x.view(torch.int16), ci, wpk, None, co, n, n, n, True, out.view(torch.int16))
    ms, cnt = capi.profile_read()["conv3d"]
    capi.profile(False)
    t = ms / 1e3 / max(cnt, 1)
    fl = 2.0 * n ** 3 * 27 * ci * co
    print(json.dumps({"conv": f"{n}^3 x {ci}->{co}", "form": args.conv_form, "ms": 1e3 * t, "tflops": fl / t / 1e12,
                      "launches": cnt}))


# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--histories", type=int, default=None, help="override histories per rank (profiling only)")
    ap.add_argument("--workload", default="ct", choices=["ct", "slab"],
                    help="headline workload (slab: the 10x10 one, for profiling only)")
    ap.add_argument("--ref-sample", type=int, default=40_000)
    ap.add_argument("--queue-depth", type=int, default=1 << 26,
                    help="primaries per transport pass of the 30x30 CT and 10x10 tallies (psl_tally_set_queue_depth; "
                         "2^26 holds a 103 GB transport workspace: fewer, longer passes)")
    ap.add_argument("--conv", nargs=3, type=int, metavar=("N", "CI", "CO"),
                    help="only time the denoiser's tensor-core convolution (profiling)")
    ap.add_argument("--conv-form", type=int, default=0, choices=[0, 1, 2],
                    help="psl_conv3d_form for --conv: 0 halo/TMA (default), 1 gather, 2 per-tap TMA")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-imrt", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-apr", action="store_true")
    ap.add_argument("--no-methods", action="store_true")
    ap.add_argument("--no-t1pct", action="store_true")
    ap.add_argument("--no-denoise", action="store_true")
    ap.add_argument("--no-slab", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.conv:
        conv_only(args)
        return

    import torch
    import torch.distributed as dist

    from paper_1302_1861_b300 import capi, engine, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c = Ctx(torch, dist, capi, engine, inputs, rank, world, local, args)

    w = headline_workload() if args.workload == "ct" else inputs.config2()
    # cpu baseline before any heavy GPU work (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.ref_sample)

    h = measure(c, w, args.steps, args.warmup, not args.no_e2e, not args.no_t1pct, not args.no_plain, profile=True)
    prof, counts, per_rank, t_step = h["prof"], h["counts"], h["per_rank"], h["t_step"]
    atom_peak = capi.atomic_peak(int(np.prod(w.phantom.shape)), 1 << 30)

    # roofline of the dominant kernel (largest device time in the timed region)
    peaks, pk_kind = measured_peaks()
    name, (ms_tot, nl) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_s = ms_tot / 1e3 / max(nl, 1)
    roof = roofline_for(name, per_launch_s, nl, args.steps, w, per_rank, peaks, pk_kind, counts, atom_peak)
    rooflines = rooflines_per_step(prof, args.steps, w, per_rank, peaks, counts)
    ms_e = prof["electron"][0] / args.steps / 1e3
    ms_p = prof["photon"][0] / args.steps / 1e3
    transport = {"electron_steps": int(counts[6]), "woodcock_steps": int(counts[10]),
                 "photon_interactions": int(counts[3] + counts[4] + counts[5]),
                 "tally_atomics": {"photon": int(counts[8]), "electron": int(counts[9])},
                 "atomics_per_s": {"photon": counts[8] / ms_p, "electron": counts[9] / ms_e},
                 "atomic_peak_per_s": atom_peak, "atomic_peak_kind": "measured: psl_atomic_peak, int64 adds into "
                                                                    f"{int(np.prod(w.phantom.shape))} cells"}
    n_counters, ws_bytes, qdepth, bps = h["tally_info"]
    del h["dw"]

    # the 10x10 workload: its own steps and measured time to 1 %
    slab = None
    if rank == 0 and world == 1 and not args.no_slab and args.workload == "ct":
        s2 = measure(c, inputs.config2(), max(3, args.steps // 2), args.warmup, False, not args.no_t1pct,
                     False)
        slab = {"workload": s2["w"].name, "value": s2["value"], "unit": "histories/s",
                "ms_per_step": 1e3 * s2["t_step"], "time_to_1pct": s2["t1pct"],
                "energy_balance": s2["energy_balance"]}
        del s2
    imrt = None
    if rank == 0 and world == 1 and not args.no_imrt:
        imrt = imrt_run(capi, engine, inputs, torch, w.records if w.index == 3 else None)
    apr = None
    if rank == 0 and world == 1 and not args.no_apr:
        apr = apr_build(capi, engine, inputs, torch, c.flush)
    denoised = None
    if rank == 0 and world == 1 and not args.no_denoise:
        measured_1pct = {w.name: h["t1pct"] if h["t1pct"].get("kind") == "measured" else None}
        if slab and slab["time_to_1pct"].get("kind") == "measured":
            measured_1pct["psl-10x10-slab64"] = slab["time_to_1pct"]
        denoised = denoised_run(capi, torch, c.flush, peaks_for_denoise(), measured_1pct)
    methods = None
    if rank == 0 and world == 1 and not args.no_methods:
        w2 = inputs.config2()
        methods = stream_method_run(capi, engine, torch, c.flush, w2, engine.upload(w2), w2.n_histories)
        if slab:
            methods["method3_psl_histories_per_s"] = slab["value"]

    if rank == 0:
        line = {"metric": METRIC, "value": h["value"], "unit": "histories/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded 6 MV-like phase space, CT-like phantom)",
                "config": workload_config(w, per_rank, world),
                "e2e": h.get("e2e"), "roofline": roof, "rooflines": rooflines, "cpu_baseline": cpu,
                "clocks": h["clocks"], "gpu_launches": int(h["launches"]),
                "time_to_1pct": h["t1pct"],
                "energy_balance": h["energy_balance"],
                "ledger_mev": {"emitted": h["ledger_mev"][0], "escaped": h["ledger_mev"][1],
                               "deposited": h["ledger_mev"][2],
                               "note": "one dose of all ranks' histories (int64 tallies summed over ranks)"},
                "transport": transport,
                "tally_memory": {"counters": n_counters, "workspace_bytes": ws_bytes, "queue_depth": qdepth,
                                 "blocks_per_sm": bps},
                "modes": {"batched_psl_run": h["value"], "plain_per_batch": h.get("plain"), "unit": "histories/s"},
                "workload_10x10": slab,
                "imrt_batched_graph": imrt,
                "apr_build": apr,
                "methods": methods,
                "denoised": denoised,
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# Per-event figures of the transport kernels, measured with ncu on one step
# of the headline workload (every k_photon / k_electron launch of the step,
# smsp__thread_inst_executed.sum over the step's Woodcock / electron steps;
# dram__bytes_read.sum + dram__bytes_write.sum per history, also for the
# source kernel):
#   ncu --metrics smsp__thread_inst_executed.sum,smsp__inst_executed.sum,gpu__time_duration.sum
#       -k regex:"k_electron|k_photon" python bench.py --steps 1 --warmup 0 --no-...
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       -k regex:"k_electron|k_photon|k_source" (the same command)
# They hold for the kernels they were measured on; re-measure after changing
# the kernels.
THREAD_INST_PER_ELECTRON_STEP = 515.3
THREAD_INST_PER_WOODCOCK_STEP = 331.9
DRAM_BYTES_PER_HISTORY = {"electron": 22.1, "photon": 57.0, "source": 77.9}
# issue speed of light: 148 SMs x 4 schedulers x 1 warp-instruction/clk x 32 lanes x 2.032 GHz
THREAD_INST_PEAK = 148 * 4 * 32 * 2.032e9


def peaks_for_denoise():
    peaks, kind = measured_peaks()
    return peaks, kind


def conv_flops(V):
    """Multiply-add FLOPs of the denoiser's convolutions on a volume of V voxels."""
    lay = [(0, 8, 16), (0, 16, 16), (1, 16, 32), (2, 32, 64), (3, 64, 128), (3, 128, 64), (2, 64, 32), (1, 32, 16),
           (0, 16, 16)]
    return sum(2.0 * (V / 8 ** lev) * 27 * ci * co for lev, ci, co in lay)


def denoised_run(capi, torch, flush, peaks, measured_1pct=None):
    """The denoised form: trained weights (the package's
    weights/denoiser_psl.npy, trained by `python -m
    paper_1302_1861_b300.denoiser` on pairs the method generated on other
    seeded geometries); on the 10x10 slab and the 30x30 CT workloads, a
    plain 4e9-history reference, low-history runs denoised and scored in the
    body, beside the plain run to 1 % (measured on whole plans by the
    headline and 10x10 legs when given, else extrapolated from the
    reference); the tensor-core convolution timed alone on its heaviest
    shape, and the network's inference on a full 128^3 volume."""
    from paper_1302_1861_b300 import denoiser as dz
    path = os.path.join(ROOT, "paper_1302_1861_b300", "weights", "denoiser_psl.npy")
    if not os.path.exists(path):
        return {"unavailable": "no trained weights"}
    den = dz.load(path)
    held_out = dz.held_out_report(den, log=None, plain_1pct=measured_1pct)
    # the convolution kernel alone: 128^3 voxels, 128 -> 128 channels (1.9e12 FLOP)
    V, ci, co = 128 ** 3, 128, 128
    x = torch.randn(V * ci, device="cuda").to(torch.bfloat16)
    wt = torch.randn(27 * ci * co, device="cuda") * 0.05
    wpk = capi.conv3d_pack(wt, ci, co)
    out = torch.empty(V * co, dtype=torch.bfloat16, device="cuda")
    for it in range(2):                                   # warm-up
        capi.conv3d(x.view(torch.int16), ci, wpk, None, co, 128, 128, 128, True, out.view(torch.int16))
    capi.profile(True)
    for it in range(4):
        flush.fill_(1.0)
        capi.conv3d(x.view(torch.int16), ci, wpk, None, co, 128, 128, 128, True, out.view(torch.int16))
    ms_conv, n_conv = capi.profile_read()["conv3d"]
    capi.profile(False)
    t_conv = ms_conv / 1e3 / max(n_conv, 1)
    fl = 2.0 * V * 27 * ci * co
    pk = peaks[0].get("bf16_tflops") if isinstance(peaks[0], dict) else None
    conv = {"shape": "128^3 x 128->128, 3x3x3", "flop": fl, "ms": 1e3 * t_conv, "tflops": fl / t_conv / 1e12,
            "peak_tflops": pk, "frac": (fl / t_conv / 1e12 / pk) if pk else None,
            "peak_kind": f"bf16_tflops ({peaks[1]}, burst: the kernel is timed alone)",
            "note": "device time of the kernel launch (the library's CUDA events on its stream), L2 flushed "
                    "before each of 4 launches"}
    # inference on a full 128^3 volume
    n = 128
    dose = torch.rand(n ** 3, device="cuda")
    rho = torch.ones(n ** 3, device="cuda")
    o = torch.empty_like(dose)
    ti = []
    for it in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        den.forward(dose, rho, n, n, n, 1.0, o)
        torch.cuda.synchronize()
        if it >= 2:
            ti.append(time.perf_counter() - t0)
    t_inf = float(np.median(ti))
    den.close()
    return {"workloads": held_out, "conv_kernel": conv,
            "inference_128cubed": {"ms": 1e3 * t_inf, "conv_tflops": conv_flops(n ** 3) / t_inf / 1e12}}


def time_to_1pct(capi, torch, w, dw, phys, n_est, sl, shape, queue_depth=None):
    """Wall time of a whole plan (psl_build, psl_plan_create, psl_run of all
    batches, dose_readout) of N histories whose isocentre uncertainty (mean
    sigma/D over the 3x3x3 voxels at the isocentre, N_b = 10 batches) is at
    most 1 %.  N starts 5 % above the estimate and grows until it holds."""
    from paper_1302_1861_b300 import engine
    nvox = dw.mat_t.numel()
    dose = torch.empty(nvox, dtype=torch.float64, device="cuda")
    sigma = torch.empty_like(dose)
    lg = torch.empty(3, dtype=torch.float64, device="cuda")
    n = int(n_est * 1.05)
    tries = []
    for _ in range(3):
        tally = capi.psl_tally_create(dw.phantom, w.n_batches)
        if queue_depth:
            capi.psl_tally_set_queue_depth(tally, queue_depth)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        store = capi.psl_build(dw.params, dw.records)
        plan = capi.psl_plan_create(store, dw.beams, w.sad, n, w.seed)
        capi.psl_run(plan, dw.phantom, phys, tally, 0, n)
        _, n_total, _ = plan.info()
        capi.dose_readout(tally, dw.phantom, engine.normalisation(plan, n),
                          dose, sigma, lg)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        d = dose.view(*shape).cpu().numpy()
        s = sigma.view(*shape).cpu().numpy()
        rel = float((s[sl] / d[sl]).mean())
        tries.append({"histories": n, "seconds": secs, "isocentre_rel_sigma": rel})
        tally.close(); plan.close(); store.close()
        if rel <= 0.01:
            return {"histories": n, "seconds": secs, "isocentre_rel_sigma": rel, "kind": "measured",
                    "histories_per_s": n / secs, "tries": tries}
        n = int(n * (rel / 0.01) ** 2 * 1.02)
    return {"histories": None, "seconds": None, "kind": "measured: not reached in 3 tries", "tries": tries}


def stream_method_run(capi, engine, torch, flush, w, dw, n, capacity=1 << 20):
    """Method 2 of the paper (Sec. 2.2) on the same workload: the phase space
    read as an unsorted stream (history h reads record h mod N), jaw model,
    on-the-fly type/energy binning in groups of `capacity`, transport and
    readout; one warm-up run, then one timed run."""
    tally = capi.psl_tally_create(dw.phantom, 1)
    nvox = dw.mat_t.numel()
    dose = torch.empty(nvox, dtype=torch.float64, device="cuda")
    sigma = torch.empty_like(dose)
    lg = torch.empty(3, dtype=torch.float64, device="cuda")
    out = {}
    for it in range(2):
        capi.psl_tally_reset(tally)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        batch = capi.psl_stream_bin(dw.records, w.binning.e_edges, dw.beams[0], capi.METHOD_JAW_MODEL, w.z_psl,
                                    w.sad, dw.phantom, 0, n, w.seed, capacity)
        e1.record()
        capi.transport_run(dw.phantom, capi.physics(), batch, tally, 0)
        capi.dose_readout(tally, dw.phantom, 1.0 / n, dose, sigma, lg)
        e2.record()
        torch.cuda.synchronize()
        groups, kept, _, _ = capi.psl_stream_info(batch)
        batch.close()
        out = {"method2_histories_per_s": n / (e0.elapsed_time(e2) / 1e3), "method2_bin_ms": e0.elapsed_time(e1),
               "method2_total_ms": e0.elapsed_time(e2), "histories": n, "groups": groups, "kept": kept,
               "capacity": capacity}
    tally.close()
    return out


def apr_build(capi, engine, inputs, torch, flush, k=4):
    """Commissioning with azimuthal redistribution (Sec. 2.3.1): psl_build of
    the 1e7-record phase space with k copies per record (k x 1e7 rotated,
    sorted records), timed with CUDA events after one warm-up build."""
    w = inputs.config2(n_histories=1000)
    w.binning.apr_copies, w.binning.apr_seed = k, 0x5EED
    dw = engine.upload(w)
    capi.psl_build(dw.params, dw.records).close()
    times = []
    for _ in range(3):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        store = capi.psl_build(dw.params, dw.records)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        n_records, n_valid, _ = store.info()
        store.close()
    t = float(np.median(times))
    return {"copies": k, "records_in": w.records.n, "records_sorted": int(n_records), "records_kept": int(n_valid),
            "ms": 1e3 * t, "sorted_records_per_s": n_records / t}


def imrt_run(capi, engine, inputs, torch, records=None):
    """The batched IMRT plan (7 gantry angles x 10-60 segments, per-segment
    fluence, 4e7-record phase space, 128x128x100 CT-like phantom, 5e8
    histories) as one CUDA-graph launch of psl_run: the persistent grid and
    queue depth picked by psl_autotune on 2e7 probe histories of the plan,
    then capture once and time the replays."""
    w = inputs.config4(records=records)
    dw = engine.upload(w)
    phys = capi.physics()
    # PSL bin size first (the store is rebuilt per candidate), then the
    # persistent grid and queue depth on the chosen store
    cells = [0.5, 1.0, 2.0]
    t0 = time.perf_counter()
    cell, cell_secs = capi.psl_autotune_bins(dw.params, dw.records, dw.beams, w.sad, dw.phantom, phys,
                                             w.n_histories, w.seed, w.n_batches, cells, 20_000_000)
    t_bins = time.perf_counter() - t0
    if cell != 1.0:
        w.binning = inputs.make_binning(20.0, cell, 32, log_ebins=True)
        dw = engine.upload(w, records=dw.rec_t)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, w.n_batches)
    t0 = time.perf_counter()
    tuned_grid, tuned_depth = capi.psl_autotune(plan, dw.phantom, phys, tally, 20_000_000)
    t_tune = time.perf_counter() - t0
    capi.psl_run(plan, dw.phantom, phys, tally, 0, w.n_histories, use_graph=True)     # capture + first run
    times = []
    for _ in range(2):
        capi.psl_tally_reset(tally)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        capi.psl_run(plan, dw.phantom, phys, tally, 0, w.n_histories, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    nz, ny, nx = w.phantom.shape
    dose = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    sigma = torch.empty_like(dose)
    lg = torch.empty(3, dtype=torch.float64, device="cuda")
    n_entries, n_total, _ = plan.info()
    capi.dose_readout(tally, dw.phantom, engine.normalisation(plan, w.n_histories), dose, sigma, lg)
    # the whole per-plan sequence (tally reset, run, readout) as one graph launch
    norm = engine.normalisation(plan, w.n_histories)
    capi.psl_plan_replay(plan, dw.phantom, phys, tally, 0, w.n_histories, norm, dose, sigma, lg)   # capture
    t_whole = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        capi.psl_plan_replay(plan, dw.phantom, phys, tally, 0, w.n_histories, norm, dose, sigma, lg)
        e1.record()
        torch.cuda.synchronize()
        t_whole.append(e0.elapsed_time(e1) / 1e3)
    d = dose.view(nz, ny, nx).cpu().numpy()
    sg = sigma.view(nz, ny, nx).cpu().numpy()
    ic = ((np.array(w.beams[0].iso) - np.array(w.phantom.origin)) / np.array(w.phantom.voxel)).astype(int)[::-1]
    sl = tuple(slice(c - 1, c + 2) for c in ic)
    rel = float((sg[sl] / d[sl]).mean())
    t = float(np.mean(times))
    rate = w.n_histories / t
    n1 = w.n_histories * (rel / 0.01) ** 2
    lgh = lg.cpu().numpy()
    tally.close(); plan.close(); store.close()
    # measured: a whole plan of N histories (psl_build to dose_readout, no
    # graph), N from the sigma above, raised until the criterion holds
    t1 = time_to_1pct(capi, torch, w, dw, phys, n1, sl, (nz, ny, nx), tuned_depth)
    return {"workload": w.name, "segments": len(w.beams), "psl_entries": n_entries, "histories": w.n_histories,
            "seconds_per_plan": t, "histories_per_s": rate, "launch": "one CUDA graph (psl_run, use_graph=1)",
            "autotuned": {"blocks_per_sm": tuned_grid, "queue_depth": tuned_depth, "probe_histories": 20_000_000,
                          "seconds": t_tune, "psl_cell_cm": cell,
                          "psl_cell_estimates_s": dict(zip(map(str, cells), map(float, cell_secs))),
                          "psl_cell_seconds": t_bins},
            "whole_plan_graph_s": float(np.mean(t_whole)),
            "whole_plan_graph": "psl_plan_replay: tally reset + all segments + dose readout in one CUDA graph launch",
            "isocentre_rel_sigma": rel, "time_to_1pct_s": n1 / rate, "time_to_1pct_s_kind": "extrapolated",
            "time_to_1pct_measured": t1,
            "energy_balance": float((lgh[1] + lgh[2] - lgh[0]) / lgh[0])}


def rooflines_per_step(prof, steps, w, per_rank, peaks, counts):
    """Every timed kernel class against its own bound, from its device time
    per step: algorithmic bytes per step over that time for the HBM-bound
    ones (the onesweep class also holds the plan's small sorts, whose bytes
    are left out; the band sort's bytes depend on the electron count, which
    the ledger does not hold), events per second against the issue speed of
    light for the transport kernels."""
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    n = w.records.n
    n_bins = 2 * w.binning.n_ebins * w.binning.nx * w.binning.ny
    passes = -(-int(np.ceil(np.log2(n_bins + 1))) // 8)     # 8-bit digits of the PSL id (+ sentinel)
    nvox = int(np.prod(w.phantom.shape))
    # gather class: k_pack (25 B read, 32 B written) + k_gather (4 B permutation,
    # 32 B record read, 32 B written) per record
    bytes_per_step = {"key": n * 17.0, "onesweep": passes * n * 16.0, "gather": n * 125.0,
                      "source": per_rank * 80.0, "readout": nvox * (w.n_batches * 8.0 + 16.0)}
    out = {}
    for k, (ms_k, n_k) in prof.items():
        if not n_k:
            continue
        t = ms_k / 1e3 / max(steps, 1)
        if k in bytes_per_step:
            a = bytes_per_step[k] / t / 1e9
            out[k] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm}
        elif k in ("electron", "photon"):
            ev, ipe = (counts[6], THREAD_INST_PER_ELECTRON_STEP) if k == "electron" else \
                (counts[10], THREAD_INST_PER_WOODCOCK_STEP)
            a, pk = ev / t / 1e9, THREAD_INST_PEAK / ipe / 1e9
            out[k] = {"bound": "alu", "achieved": a, "peak": pk, "unit": "Gevents/s", "frac": a / pk}
    return out


def roofline_for(name, per_launch_s, launches, steps, w, per_rank, peaks, pk_kind, counts, atom_peak=None):
    """Algorithmic bytes (HBM-bound kernels) or operations per launch over the
    measured launch duration."""
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    n = w.records.n
    per_step = max(launches // max(steps, 1), 1)
    if name in ("onesweep", "key", "gather", "source", "band_sort", "readout"):
        if name == "onesweep":
            byts = n * 16.0                          # read key+value, write key+value
        elif name == "key":
            byts = n * (13.0 + 4.0)                  # read x, y, e, q; write the PSL id
        elif name == "gather":
            byts = n * 125.0 / 2.0                   # k_pack + k_gather (see rooflines_per_step), per launch
        elif name == "source":
            byts = per_rank / per_step * (32.0 + 48.0)
        elif name == "readout":
            nvox = int(np.prod(w.phantom.shape))
            byts = nvox * (w.n_batches * 8.0 + 16.0)  # the batch tallies read, dose and sigma written
        else:
            byts = 0.0
        ach = byts / per_launch_s / 1e9
        traffic = DRAM_BYTES_PER_HISTORY[name] * per_rank / per_step if name in DRAM_BYTES_PER_HISTORY else None
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "peak_kind": pk_kind, "launches": launches}
    # transport: events per second against the instruction-issue speed of light
    per_step = max(launches // max(steps, 1), 1)
    if name == "electron":
        events, ipe = counts[6], THREAD_INST_PER_ELECTRON_STEP
    else:
        events, ipe = counts[10], THREAD_INST_PER_WOODCOCK_STEP
    ach = events / per_step / per_launch_s / 1e9
    peak = THREAD_INST_PEAK / ipe / 1e9 if ipe else None
    traffic = DRAM_BYTES_PER_HISTORY.get(name, 0.0) * per_rank / per_step
    # the tally's bound: the kernel's int64 atomics per second against the
    # measured int64 atomic peak (psl_atomic_peak)
    at = counts[9] if name == "electron" else counts[8]
    atomic = None
    if atom_peak:
        a_rate = at / per_step / per_launch_s
        atomic = {"achieved": a_rate, "peak": atom_peak, "unit": "int64 atomics/s", "frac": a_rate / atom_peak}
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gevents/s",
            "frac": ach / peak if peak else None, "traffic": traffic, "per_launch_ms": per_launch_s * 1e3,
            "atomic_bound": atomic,
            "launches": launches, "events": "electron steps" if name == "electron" else "Woodcock steps",
            "events_per_launch": events / per_step,
            "peak_kind": "derived: 148 SMs x 4 issue/clk x 32 lanes x 2.032 GHz / %.1f thread instructions "
                         "per event (ncu)" % ipe,
            "traffic_kind": "ncu dram bytes of all the kernel's launches in one step of this workload, "
                            "per history, times the histories per launch"}


if __name__ == "__main__":
    main()
