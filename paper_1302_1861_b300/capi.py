"""Thin ctypes binding of the C ABI in include/psl.h (argument marshalling only).

Every step of the path runs in libpsl_b300.so; this module only turns torch
tensors into device pointers, Python numbers into C structs and status codes
into exceptions.  It never falls back to anything else: if the library is
missing or CUDA is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PSL_B300_LIB") or os.path.join(HERE, "libpsl_b300.so")

PSL_OK, PSL_EINVAL, PSL_ENOMEM, PSL_ECUDA, PSL_ETIMEOUT, PSL_EOVERFLOW = 0, -1, -2, -3, -4, -5
PHYS_LOCAL_SECONDARIES, PHYS_FIRST_INTERACTION, PHYS_NO_MSC, PHYS_NO_HARD = 1, 2, 4, 8
SRC_TRANSPORT, SRC_JAW, SRC_FLUENCE, SRC_ZERO_WEIGHT, SRC_MISS = 0, 1, 2, 3, 4

EXPORTS = (
    "psl_physics_default", "psl_build", "psl_store_info", "psl_store_read", "psl_plan_create",
    "psl_plan_info", "psl_plan_read", "psl_source_batch", "psl_source_trace", "psl_batch_from_particles",
    "psl_batch_info", "psl_tally_create", "psl_tally_reset", "psl_tally_read", "transport_run",
    "transport_trace", "dose_readout", "psl_store_destroy", "psl_plan_destroy", "psl_batch_destroy",
    "psl_tally_destroy", "psl_last_error", "psl_kernel_launches", "psl_profile", "psl_profile_read",
    "psl_build_static", "psl_atomic_peak", "psl_run", "psl_autotune", "psl_stream_bin", "psl_stream_info",
    "psl_stream_read", "psl_batch_read", "psl_memory_trim",
    "psl_conv3d_packed_size", "psl_conv3d_pack", "psl_conv3d", "psl_conv3d_wgrad", "psl_denoiser_param_count",
    "psl_denoiser_create", "psl_denoiser_destroy", "psl_denoiser_params", "psl_denoiser_forward",
    "psl_denoiser_backward", "psl_denoiser_step", "psl_gamma", "psl_conv3d_form", "psl_tally_set_order",
    "psl_kth_smallest", "psl_tally_buffers", "psl_tally_info", "psl_tally_set_queue_depth",
    "psl_dose_normalisation", "psl_tally_trace_source", "psl_debug_waits", "psl_plan_replay",
    "psl_autotune_bins",
)
METHOD_PATIENT_DEPENDENT, METHOD_JAW_MODEL = 1, 2
SLICE_BY_HISTORY, MAX_BATCHES = -1, 1024
ORDER_AUTO, ORDER_READING, ORDER_BATCH = 0, 1, 2
STATIC_MAX_RECORDS = 1 << 20
DEBUG_LOOKBACK_STALL, DEBUG_FEED_STALL = 1, 2

vp = ctypes.c_void_p
f32, i32, i64, u32, u64, f64 = (ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_double)


class Records(ctypes.Structure):
    _fields_ = [("x", vp), ("y", vp), ("u", vp), ("v", vp), ("e", vp), ("wt", vp), ("q", vp), ("n", i64)]


class Params(ctypes.Structure):
    _fields_ = [("nx", i32), ("ny", i32), ("n_ebins", i32), ("apr_copies", i32), ("x_edges", vp),
                ("y_edges", vp), ("e_edges", vp), ("z_psl", f32), ("apr_seed", ctypes.c_uint64)]


class Beam(ctypes.Structure):
    _fields_ = [("x1", f32), ("x2", f32), ("y1", f32), ("y2", f32), ("z_jaw_x", f32), ("z_jaw_y", f32),
                ("gantry", f32), ("collimator", f32), ("couch", f32), ("mu", f32), ("roi_margin", f32),
                ("iso", f32 * 3), ("fnx", i32), ("fny", i32), ("fx0", f32), ("fy0", f32), ("fdx", f32),
                ("fdy", f32), ("fluence", vp)]


class Phantom(ctypes.Structure):
    _fields_ = [("nx", i32), ("ny", i32), ("nz", i32), ("vx", f32), ("vy", f32), ("vz", f32),
                ("origin", f32 * 3), ("mat", vp), ("rho", vp)]


class Physics(ctypes.Structure):
    _fields_ = [("photon_cut", f32), ("electron_cut", f32), ("wcc", f32), ("wcb", f32), ("flags", u32)]


class PslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"PSL error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libpsl_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built: run python -m paper_1302_1861_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name in EXPORTS:
            getattr(L, name)
        L.psl_kernel_launches.restype = ctypes.c_int64
        L.psl_kernel_launches.argtypes = []
        L.psl_last_error.restype = ctypes.c_char_p
        L.psl_last_error.argtypes = []
        L.psl_denoiser_param_count.restype = ctypes.c_int64
        L.psl_denoiser_param_count.argtypes = []
        L.psl_denoiser_destroy.restype = None
        L.psl_denoiser_destroy.argtypes = [vp]
        L.psl_conv3d_packed_size.restype = ctypes.c_int64
        L.psl_conv3d_packed_size.argtypes = [i32, i32]
        L.psl_physics_default.restype = None
        L.psl_physics_default.argtypes = [vp]
        for name in ("psl_store_destroy", "psl_plan_destroy", "psl_batch_destroy", "psl_tally_destroy"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [vp]
        sig = {
            "psl_build": [vp, vp, vp, vp],
            "psl_build_static": [vp, vp, vp, vp, vp, vp],
            "psl_store_info": [vp, vp, vp, vp],
            "psl_store_read": [vp, vp, vp, vp, vp],
            "psl_plan_create": [vp, vp, i32, f32, i64, u64, vp, vp],
            "psl_plan_info": [vp, vp, vp, vp],
            "psl_plan_read": [vp, vp, vp, vp, vp, vp],
            "psl_source_batch": [vp, vp, i64, i64, i64, vp, vp],
            "psl_source_trace": [vp, vp, i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp],
            "psl_batch_from_particles": [vp, vp, vp, i64, u64, vp, vp],
            "psl_batch_info": [vp, vp, vp, vp],
            "psl_tally_create": [vp, i32, vp],
            "psl_tally_reset": [vp, vp],
            "psl_tally_read": [vp, vp, vp, vp],
            "transport_run": [vp, vp, vp, vp, i32, vp],
            "transport_trace": [vp, vp, vp, vp, i32, vp, vp, vp, vp],
            "dose_readout": [vp, vp, f64, vp, vp, vp, vp],
            "psl_profile": [ctypes.c_int],
            "psl_atomic_peak": [i64, i64, vp, vp],
            "psl_run": [vp, vp, vp, vp, i64, i64, i32, vp],
            "psl_autotune": [vp, vp, vp, vp, i64, vp, vp, vp],
            "psl_profile_read": [i32, vp, vp, vp],
            "psl_stream_bin": [vp, vp, i32, vp, i32, f32, f32, vp, i64, i64, u64, i64, vp, vp],
            "psl_stream_info": [vp, vp, vp, vp, vp],
            "psl_stream_read": [vp, vp, vp, vp, vp],
            "psl_batch_read": [vp, vp, vp, vp, vp],
            "psl_memory_trim": [u64, vp],
            "psl_conv3d_pack": [vp, i32, i32, i32, vp, vp],
            "psl_conv3d": [vp, i32, vp, vp, i32, i32, i32, i32, i32, vp, vp, vp],
            "psl_conv3d_wgrad": [vp, i32, vp, i32, i32, i32, i32, vp, vp],
            "psl_denoiser_create": [u64, vp],
            "psl_denoiser_params": [vp, vp, vp, vp, vp],
            "psl_denoiser_forward": [vp, vp, vp, i32, i32, i32, f32, vp, vp],
            "psl_denoiser_backward": [vp, vp, vp, vp, i32, i32, i32, f32, vp, vp],
            "psl_denoiser_step": [vp, f32, vp],
            "psl_gamma": [vp, vp, i32, i32, i32, f32, f32, f32, f64, f64, f64, i32, f64, vp, vp, vp],
            "psl_conv3d_form": [i32],
            "psl_tally_set_order": [vp, i32],
            "psl_kth_smallest": [vp, i64, i64, vp, vp],
            "psl_tally_buffers": [vp, vp, vp],
            "psl_tally_info": [vp, vp, vp, vp, vp],
            "psl_tally_set_queue_depth": [vp, i64],
            "psl_dose_normalisation": [vp, i64, i64, f64, vp],
            "psl_tally_trace_source": [vp, i64, i64, vp, vp, vp, vp, vp, vp],
            "psl_debug_waits": [i64, u32, i64],
            "psl_plan_replay": [vp, vp, vp, vp, i64, i64, f64, vp, vp, vp, vp],
            "psl_autotune_bins": [vp, vp, vp, i32, f32, vp, vp, i64, u64, i32, vp, i32, i64, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int):
    if code != PSL_OK:
        raise PslError(code, lib().psl_last_error().decode())


def ptr(t) -> Optional[int]:
    """Device (or host) address of a torch tensor / numpy array; None passes NULL."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def stream_ptr(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def kernel_launches() -> int:
    return int(lib().psl_kernel_launches())


PSL_NK = 9


def atomic_peak(n_cells: int, n_updates: int = 1 << 30, stream=None) -> float:
    """Measured int64 atomic-add throughput (updates/s) into n_cells counters."""
    v = f64()
    check(lib().psl_atomic_peak(int(n_cells), int(n_updates), ctypes.byref(v), stream_ptr(stream)))
    return v.value


def profile(enable: bool):
    check(lib().psl_profile(1 if enable else 0))


def profile_read():
    """{kernel name: (total ms, launches)} of the timed launches."""
    out = {}
    for k in range(PSL_NK):
        ms, n, name = f64(), i64(), ctypes.c_char_p()
        check(lib().psl_profile_read(k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(name)))
        out[name.value.decode()] = (ms.value, n.value)
    return out


def physics(flags: int = 0, **kw) -> Physics:
    p = Physics()
    lib().psl_physics_default(ctypes.byref(p))
    p.flags = flags
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Handle:
    """Owns a library handle and destroys it with the matching call."""
    _destroy = None

    def __init__(self, h: int):
        self.h = ctypes.c_void_p(h)

    def close(self):
        if self.h and self.h.value:
            getattr(lib(), self._destroy)(self.h)
            self.h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Store(Handle):
    _destroy = "psl_store_destroy"

    def info(self):
        a, b, c = i64(), i64(), i64()
        check(lib().psl_store_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


class Plan(Handle):
    _destroy = "psl_plan_destroy"

    def info(self):
        a, b, c = i64(), i64(), i64()
        check(lib().psl_plan_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


class Batch(Handle):
    _destroy = "psl_batch_destroy"

    def info(self):
        a, b, c = i64(), i64(), i64()
        check(lib().psl_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


class Tally(Handle):
    _destroy = "psl_tally_destroy"


def _out_handle():
    return ctypes.c_void_p(0)


def psl_build(params: Params, records: Records, stream=None) -> Store:
    h = _out_handle()
    check(lib().psl_build(ctypes.byref(params), ctypes.byref(records), ctypes.byref(h), stream_ptr(stream)))
    return Store(h.value)


def psl_build_static(params: Params, records: Records, offsets, sorted_records, stream=None) -> int:
    """PSL build into caller arrays with no device allocation (see psl.h);
    returns the number of records kept."""
    nv = i64()
    check(lib().psl_build_static(ctypes.byref(params), ctypes.byref(records), ptr(offsets), ptr(sorted_records),
                                 ctypes.byref(nv), stream_ptr(stream)))
    return nv.value


def psl_store_read(store: Store, offsets=None, perm=None, records=None, stream=None):
    check(lib().psl_store_read(store.h, ptr(offsets), ptr(perm), ptr(records), stream_ptr(stream)))


def psl_plan_create(store: Store, beams: Sequence[Beam], sad: float, n_histories: int, seed: int,
                    stream=None) -> Plan:
    arr = (Beam * len(beams))(*beams)
    h = _out_handle()
    check(lib().psl_plan_create(store.h, arr, len(beams), sad, int(n_histories), int(seed), ctypes.byref(h),
                                stream_ptr(stream)))
    return Plan(h.value)


def psl_plan_read(plan: Plan, beam=None, psl=None, count=None, offset=None, stream=None):
    check(lib().psl_plan_read(plan.h, ptr(beam), ptr(psl), ptr(count), ptr(offset), stream_ptr(stream)))


def psl_source_batch(plan: Plan, phantom: Phantom, first: int, n: int, stride: int = 1, stream=None) -> Batch:
    h = _out_handle()
    check(lib().psl_source_batch(plan.h, ctypes.byref(phantom), int(first), int(n), int(stride), ctypes.byref(h),
                                 stream_ptr(stream)))
    return Batch(h.value)


def psl_source_trace(plan: Plan, phantom: Phantom, first: int, n: int, entry=None, use=None, rec=None,
                     beam=None, status=None, state=None, ptype=None, stride: int = 1, stream=None):
    check(lib().psl_source_trace(plan.h, ctypes.byref(phantom), int(first), int(n), int(stride), ptr(entry), ptr(use),
                                 ptr(rec), ptr(beam), ptr(status), ptr(state), ptr(ptype), stream_ptr(stream)))


def psl_batch_from_particles(state, ptype, pid, seed: int, stream=None) -> Batch:
    h = _out_handle()
    check(lib().psl_batch_from_particles(ptr(state), ptr(ptype), ptr(pid), int(ptype.shape[0]), int(seed),
                                         ctypes.byref(h), stream_ptr(stream)))
    return Batch(h.value)


def psl_stream_bin(records: Records, e_edges, beam: Beam, method: int, z_psl: float, sad: float, phantom: Phantom,
                   first: int, n: int, seed: int, capacity: int, stream=None) -> Batch:
    """Methods 1 / 2: the on-the-fly type/energy binning of the phase-space
    stream (see psl.h); e_edges is a host float32 array."""
    ee = np.ascontiguousarray(e_edges, np.float32)
    h = _out_handle()
    check(lib().psl_stream_bin(ctypes.byref(records), ee.ctypes.data, int(len(ee) - 1), ctypes.byref(beam),
                               int(method), float(z_psl), float(sad), ctypes.byref(phantom), int(first), int(n),
                               int(seed), int(capacity), ctypes.byref(h), stream_ptr(stream)))
    return Batch(h.value)


def psl_stream_info(batch: Batch):
    """(groups, particles kept, emitted fixed point, missed fixed point)."""
    a, b, c, d = i64(), i64(), i64(), i64()
    check(lib().psl_stream_info(batch.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def psl_stream_read(batch: Batch, group_bin=None, group_count=None, history=None, stream=None):
    check(lib().psl_stream_read(batch.h, ptr(group_bin), ptr(group_count), ptr(history), stream_ptr(stream)))


def psl_batch_read(batch: Batch, state=None, ptype=None, pid=None, stream=None):
    check(lib().psl_batch_read(batch.h, ptr(state), ptr(ptype), ptr(pid), stream_ptr(stream)))


def memory_held() -> int:
    """Bytes the library's device memory pool reserves on the current device
    (psl_memory_trim asked to keep all of it; a transport workspace kept from
    a destroyed tally is still freed)."""
    return memory_trim(keep_bytes=(1 << 64) - 1)


def memory_trim(keep_bytes: int = 0) -> int:
    """Free the transport workspace kept from a destroyed tally, then return
    the library pool's memory beyond keep_bytes to the driver; returns the
    bytes the pool still reserves."""
    held = u64()
    check(lib().psl_memory_trim(int(keep_bytes), ctypes.byref(held)))
    return held.value


def conv3d_pack(w, ci: int, co: int, mirror: bool = False, stream=None):
    """FP32 taps (device [27, ci, co]) -> packed BF16 tiles (a device int16 tensor)."""
    import torch
    cin, cout = (co, ci) if mirror else (ci, co)
    n = int(lib().psl_conv3d_packed_size(cin, cout))
    out = torch.empty(n, dtype=torch.int16, device=w.device)
    check(lib().psl_conv3d_pack(ptr(w), int(ci), int(co), 1 if mirror else 0, ptr(out), stream_ptr(stream)))
    return out


def conv3d(x, ci: int, wpk, bias, co: int, nx: int, ny: int, nz: int, relu: bool, out=None, out_f32=None,
           stream=None):
    """3x3x3 convolution on the tensor cores (see psl_denoise.h); x, out: BF16 bit patterns."""
    check(lib().psl_conv3d(ptr(x), int(ci), ptr(wpk), ptr(bias), int(co), int(nx), int(ny), int(nz),
                           1 if relu else 0, ptr(out), ptr(out_f32), stream_ptr(stream)))


def conv3d_form(form: int):
    """0: TMA form where the volume allows, 1: gather form everywhere."""
    check(lib().psl_conv3d_form(int(form)))


def conv3d_wgrad(x, ci: int, gy, co: int, nx: int, ny: int, nz: int, dw, stream=None):
    """dw[27, ci, co] (FP32, device) += the tap gradient (see psl_denoise.h)."""
    check(lib().psl_conv3d_wgrad(ptr(x), int(ci), ptr(gy), int(co), int(nx), int(ny), int(nz), ptr(dw),
                                 stream_ptr(stream)))


def gamma(ref, ev, voxel, dose_crit=0.02, dta_cm=0.2, threshold=0.10, upsample=4, max_radius_cm=0.0,
          stream=None):
    """Global gamma pass rate of ev against ref (device float64 [nz, ny, nx]);
    returns (pass rate, voxels evaluated)."""
    nz, ny, nx = ref.shape
    rate, n = ctypes.c_double(), i64()
    check(lib().psl_gamma(ptr(ref), ptr(ev), nx, ny, nz, float(voxel[0]), float(voxel[1]), float(voxel[2]),
                          float(dose_crit), float(dta_cm), float(threshold), int(upsample), float(max_radius_cm),
                          ctypes.byref(rate), ctypes.byref(n), stream_ptr(stream)))
    return rate.value, n.value


class Denoiser(Handle):
    """The dose denoiser network (see psl_denoise.h)."""
    _destroy = "psl_denoiser_destroy"

    @staticmethod
    def param_count() -> int:
        return int(lib().psl_denoiser_param_count())

    @classmethod
    def create(cls, seed: int = 0) -> "Denoiser":
        h = _out_handle()
        check(lib().psl_denoiser_create(int(seed), ctypes.byref(h)))
        return cls(h.value)

    def params(self, set=None, get=None, grad=None, stream=None):
        check(lib().psl_denoiser_params(self.h, ptr(set), ptr(get), ptr(grad), stream_ptr(stream)))

    def forward(self, dose, rho, nx: int, ny: int, nz: int, scale: float, out, stream=None):
        check(lib().psl_denoiser_forward(self.h, ptr(dose), ptr(rho), int(nx), int(ny), int(nz), float(scale),
                                         ptr(out), stream_ptr(stream)))

    def backward(self, dose, rho, target, nx: int, ny: int, nz: int, scale: float, stream=None) -> float:
        loss = ctypes.c_double()
        check(lib().psl_denoiser_backward(self.h, ptr(dose), ptr(rho), ptr(target), int(nx), int(ny), int(nz),
                                          float(scale), ctypes.byref(loss), stream_ptr(stream)))
        return loss.value

    def step(self, lr: float, stream=None):
        check(lib().psl_denoiser_step(self.h, float(lr), stream_ptr(stream)))


def psl_tally_create(phantom: Phantom, n_batches: int) -> Tally:
    h = _out_handle()
    check(lib().psl_tally_create(ctypes.byref(phantom), int(n_batches), ctypes.byref(h)))
    return Tally(h.value)


def kth_smallest(x, k: int, stream=None) -> float:
    """The k-th smallest (0-based) of the values of a float32 device tensor."""
    v = f32()
    check(lib().psl_kth_smallest(ptr(x), int(x.numel()), int(k), ctypes.byref(v), stream_ptr(stream)))
    return v.value


def psl_tally_set_order(tally: Tally, order: int):
    check(lib().psl_tally_set_order(tally.h, int(order)))


def psl_tally_buffers(tally: Tally):
    """Device addresses of the tally's int64 counters [n_batches][nvox] and ledger [12]."""
    t, g = vp(), vp()
    check(lib().psl_tally_buffers(tally.h, ctypes.byref(t), ctypes.byref(g)))
    return t.value, g.value


def psl_tally_info(tally: Tally):
    """(int64 counters, transport workspace bytes, queue depth, blocks per SM)."""
    a, b, c, d = i64(), i64(), i64(), i32()
    check(lib().psl_tally_info(tally.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def psl_tally_trace_source(tally: Tally, first: int, n: int, entry=None, use=None, rec=None, status=None,
                           state=None, ptype=None):
    """Record the production source stage's decisions for histories [first, first+n) (n = 0: off)."""
    check(lib().psl_tally_trace_source(tally.h, int(first), int(n), ptr(entry), ptr(use), ptr(rec), ptr(status),
                                       ptr(state), ptr(ptype)))


def debug_waits(polls: int = 0, flags: int = 0, queue_cap: int = 0):
    """Failure-detection hooks (tests): polls of a bounded device wait, stalls
    that make a wait run out, a cap on the particle queues; all 0 restores."""
    check(lib().psl_debug_waits(int(polls), int(flags), int(queue_cap)))


def psl_tally_set_queue_depth(tally: Tally, depth: int):
    check(lib().psl_tally_set_queue_depth(tally.h, int(depth)))


def dose_normalisation(plan: Plan, n_histories: int, n_incident: int = 0, calibration: float = 1.0) -> float:
    """Sec. 2.5 normalisation computed by the library (psl_dose_normalisation)."""
    v = f64()
    check(lib().psl_dose_normalisation(plan.h, int(n_histories), int(n_incident), float(calibration),
                                       ctypes.byref(v)))
    return v.value


def psl_tally_reset(tally: Tally, stream=None):
    check(lib().psl_tally_reset(tally.h, stream_ptr(stream)))


def psl_tally_read(tally: Tally, tallies=None, ledger=None, stream=None):
    check(lib().psl_tally_read(tally.h, ptr(tallies), ptr(ledger), stream_ptr(stream)))


def transport_run(phantom: Phantom, phys: Physics, batch: Batch, tally: Tally, batch_index: int, stream=None):
    check(lib().transport_run(ctypes.byref(phantom), ctypes.byref(phys), batch.h, tally.h, int(batch_index),
                              stream_ptr(stream)))


def transport_trace(phantom: Phantom, phys: Physics, batch: Batch, tally: Tally, batch_index: int,
                    hist_dep=None, hist_esc=None, hist_events=None, stream=None):
    check(lib().transport_trace(ctypes.byref(phantom), ctypes.byref(phys), batch.h, tally.h, int(batch_index),
                                ptr(hist_dep), ptr(hist_esc), ptr(hist_events), stream_ptr(stream)))


def dose_readout(tally: Tally, phantom: Phantom, norm: float, dose=None, sigma=None, ledger=None, stream=None):
    check(lib().dose_readout(tally.h, ctypes.byref(phantom), float(norm), ptr(dose), ptr(sigma), ptr(ledger),
                             stream_ptr(stream)))


def psl_run(plan: Plan, phantom: Phantom, phys: Physics, tally: Tally, first: int, n: int, use_graph: bool = False,
            stream=None):
    check(lib().psl_run(plan.h, ctypes.byref(phantom), ctypes.byref(phys), tally.h, int(first), int(n),
                        1 if use_graph else 0, stream_ptr(stream)))


def psl_plan_replay(plan: Plan, phantom: Phantom, phys: Physics, tally: Tally, first: int, n: int, norm: float,
                    dose=None, sigma=None, ledger=None, stream=None):
    """Tally reset + psl_run + dose_readout recorded once as a CUDA graph, then replayed."""
    check(lib().psl_plan_replay(plan.h, ctypes.byref(phantom), ctypes.byref(phys), tally.h, int(first), int(n),
                                float(norm), ptr(dose), ptr(sigma), ptr(ledger), stream_ptr(stream)))


def psl_autotune_bins(params: Params, records: Records, beams: Sequence[Beam], sad: float, phantom: Phantom,
                      phys: Physics, n_histories: int, seed: int, n_batches: int, cells, n_probe: int, stream=None):
    """PSL position-bin size autotuner: returns (best cell size, estimated seconds per candidate)."""
    arr = (Beam * len(beams))(*beams)
    c = np.ascontiguousarray(cells, np.float32)
    out = np.zeros(len(c))
    best = f32()
    check(lib().psl_autotune_bins(ctypes.byref(params), ctypes.byref(records), arr, len(beams), float(sad),
                                  ctypes.byref(phantom), ctypes.byref(phys), int(n_histories), int(seed),
                                  int(n_batches), c.ctypes.data, len(c), int(n_probe), ctypes.byref(best),
                                  out.ctypes.data, stream_ptr(stream)))
    return best.value, out


def psl_autotune(plan: Plan, phantom: Phantom, phys: Physics, tally: Tally, n_probe: int, stream=None):
    g, d = i32(), i64()
    check(lib().psl_autotune(plan.h, ctypes.byref(phantom), ctypes.byref(phys), tally.h, int(n_probe),
                             ctypes.byref(g), ctypes.byref(d), stream_ptr(stream)))
    return g.value, d.value
