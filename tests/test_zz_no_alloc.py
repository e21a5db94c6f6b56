"""The allocation-free PSL build (psl_build_static) against psl_build.

Some callers cannot call cudaMalloc: code running inside another runtime's
memory pool, under a fixed device-memory budget, or in a process that must
not allocate after start-up.  psl_build_static gives them the same PSL sort
with its scratch in a fixed device array.  Its output must equal psl_build's
bit for bit, on two calls in a row (the shared array keeps the previous
call's contents, so the second call checks that nothing stale leaks in), and
a call must leave the device's free memory and the library pool's holding
unchanged.
"""
import ctypes

import numpy as np
import pytest

from paper_1302_1861_b300 import capi, inputs


def test_static_build_rejects_sizes_beyond_its_limit():
    """Checked before any device work: no GPU needed."""
    n = capi.STATIC_MAX_RECORDS + 1
    xe = np.array([-1, 1], np.float32)
    prm = capi.Params(1, 1, 1, 1, xe.ctypes.data, xe.ctypes.data, np.array([0, 1], np.float32).ctypes.data, 100.0)
    rec = capi.Records()
    rec.n = n
    dummy = ctypes.c_void_p(16)
    nv = ctypes.c_int64()
    rc = capi.lib().psl_build_static(ctypes.byref(prm), ctypes.byref(rec), dummy, dummy, ctypes.byref(nv), None)
    assert rc == capi.PSL_EINVAL
    assert b"exceed the static limit" in capi.lib().psl_last_error()


@pytest.mark.gpu
def test_static_build_equals_psl_build_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_1861_b300 import engine

    def memory():
        """What the library's pool holds and the device's free memory (the
        driver's count), read after a workspace kept by earlier tests is freed."""
        torch.cuda.synchronize()
        held = capi.memory_held()
        free, _ = torch.cuda.mem_get_info()
        return held, free

    # a larger input first, then a smaller one with a different binning
    for k, w in enumerate((inputs.config2(n_records=600_000, n_histories=1000), inputs.config1(n_records=90_001))):
        dw = engine.upload(w)
        n = w.records.n
        store = capi.psl_build(dw.params, dw.records)
        _, n_valid, n_bins = store.info()
        ref_off = torch.empty(n_bins + 1, dtype=torch.int64, device="cuda")
        ref_rec = torch.empty(max(n_valid, 1) * 8, dtype=torch.float32, device="cuda")
        capi.psl_store_read(store, ref_off, None, ref_rec)
        off = torch.full((n_bins + 1,), -1, dtype=torch.int64, device="cuda")
        rec = torch.full((n * 8,), -1.0, dtype=torch.float32, device="cuda")
        if k == 0:
            # the first call in the context commits the library's static array
            capi.psl_build_static(dw.params, dw.records, off, rec)
            off.fill_(-1)
            rec.fill_(-1.0)
        before = memory()
        nv = capi.psl_build_static(dw.params, dw.records, off, rec)
        after = memory()
        assert after == before, (before, after)            # no device memory taken or given back
        assert nv == n_valid
        assert torch.equal(off, ref_off)
        a = rec[: nv * 8].view(torch.int32).cpu().numpy()
        b = ref_rec[: nv * 8].view(torch.int32).cpu().numpy()
        assert np.array_equal(a, b)
