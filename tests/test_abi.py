"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/psl.h and include/psl_denoise.h declare (CPU only,
no compute calls)."""
import ctypes
import os
import re

from paper_1302_1861_b300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in ("psl.h", "psl_denoise.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"^PSL_API\s+[\w\s\*]*?\b(\w+)\(", text, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared()
    for core in ("psl_build", "psl_source_batch", "transport_run", "dose_readout"):
        assert core in names
    assert set(names) == set(capi.EXPORTS)


def test_library_exports_every_declared_symbol():
    so = build.build()
    L = ctypes.CDLL(so)
    for name in declared():
        assert hasattr(L, name), name
    # the binding's own loader resolves the same names
    capi.lib()


def test_physics_defaults_without_gpu():
    p = capi.physics()
    assert abs(p.photon_cut - 0.010) < 1e-9
    assert abs(p.electron_cut - (0.700 - 0.51099895)) < 1e-7
    assert p.wcc == p.wcb and abs(p.wcc - 0.2) < 1e-7 and p.flags == 0


def test_invalid_arguments_fail_cleanly_without_gpu():
    L = capi.lib()
    prm = capi.Params(0, 0, 0, 1, None, None, None, 100.0)
    rec = capi.Records()
    h = ctypes.c_void_p(0)
    assert L.psl_build(ctypes.byref(prm), ctypes.byref(rec), ctypes.byref(h), None) == capi.PSL_EINVAL
    assert b"bad bin counts" in L.psl_last_error()
    assert L.psl_plan_create(None, None, 0, 100.0, 10, 1, ctypes.byref(h), None) == capi.PSL_EINVAL
    assert L.psl_tally_set_order(None, capi.ORDER_BATCH) == capi.PSL_EINVAL
    # a tally of 2^33 voxels is refused before any device work (voxels are indexed in 32 bits)
    big = capi.Phantom(2048, 2048, 2048, 0.1, 0.1, 0.1, (capi.f32 * 3)(0, 0, 0), None, None)
    assert L.psl_tally_create(ctypes.byref(big), 10, ctypes.byref(h)) == capi.PSL_EINVAL
    assert b"2^31" in L.psl_last_error()
    assert L.psl_kth_smallest(None, 10, 0, None, None) == capi.PSL_EINVAL
