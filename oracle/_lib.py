"""ctypes loader of the oracle's C code: transport and stream binning
(TEST INFRASTRUCTURE).

Builds ``oracle/_build/liboracle.so`` with gcc on first use.  Only the tests,
the package smoke check and the CPU-baseline leg of the benchmark load it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "transport.c"), os.path.join(HERE, "stream.c")]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code (plain gcc, OpenMP, no FMA contraction)."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SRC)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < newest:
        tmp = SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-Wall", "-o", tmp] + SRC + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i64, u64, u32, i32, vp = (ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p)
            for name in ("ora_kn_sigma", "ora_rad_stopping"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d]
            L.ora_mu_rho.restype = d
            L.ora_mu_rho.argtypes = [d, i32, i32]
            for name in ("ora_col_stopping", "ora_moller_dcs", "ora_moller_sigma", "ora_brem_sigma",
                         "ora_bhabha_dcs", "ora_bhabha_sigma", "ora_pos_col_stopping"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d]
            for name in ("ora_restricted_stopping", "ora_restricted_stopping_pos", "ora_range", "ora_range_inv",
                         "ora_range_pos", "ora_range_inv_pos", "ora_highland"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d, d]
            L.ora_sample_bhabha.restype = None
            L.ora_sample_bhabha.argtypes = [d, d, u64, i64, vp]
            L.ora_sample_msc.restype = None
            L.ora_sample_msc.argtypes = [d, u64, i64, vp, vp]
            L.ora_sample_brem.restype = None
            L.ora_sample_brem.argtypes = [d, d, u64, i64, vp]
            L.ora_sample_pair.restype = None
            L.ora_sample_pair.argtypes = [d, u64, i64, vp, vp]
            L.ora_sample_annihilation.restype = None
            L.ora_sample_annihilation.argtypes = [u64, i64, vp, vp]
            L.ora_rotate.restype = None
            L.ora_rotate.argtypes = [i64, vp, vp, vp, vp]
            L.ora_philox.restype = None
            L.ora_philox.argtypes = [i64, vp, vp, vp]
            L.ora_sample_kn.restype = None
            L.ora_sample_kn.argtypes = [d, u64, i64, vp, vp]
            L.ora_sample_moller.restype = None
            L.ora_sample_moller.argtypes = [d, d, u64, i64, vp]
            L.ora_stream_bin.restype = i64
            L.ora_stream_bin.argtypes = [i64, vp, i32, i64, vp, vp, vp]
            L.ora_transport.restype = i32
            L.ora_transport.argtypes = ([i64] + [vp] * 6 + [i32, i32, i32, d, d, d, vp, vp, u64, u32,
                                        d, d, d, d] + [vp] * 6 + [i32])
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of each row of ctr (n x 4) under key (n x 2)."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(key, (len(ctr), 2)), np.uint32)
    out = np.zeros_like(ctr)
    lib().ora_philox(len(ctr), _p(ctr), _p(key), _p(out))
    return out
