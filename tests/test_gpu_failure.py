"""Failure detection without a GPU fault: every device-side wait is bounded
and a queue that overflows is reported, so the library returns an error
code promptly and the CUDA context stays usable.

psl_debug_waits lowers the number of polls a wait makes and makes a wait
wait on something that never comes (a flag that nothing sets): the onesweep
look-back of the PSL sort never sees its predecessors' counts, or the photon
feed's second chunk is never copied, so its mbarrier never completes.  It can
also cap the particle queues so that secondaries overflow them.  Each test
checks the status, that the call returned within seconds, and that a normal
call right after it gives the normal result.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402


@pytest.fixture(autouse=True)
def _cuda_and_reset():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    capi.debug_waits(0, 0, 0)


def _expect(code, fn):
    t0 = time.perf_counter()
    with pytest.raises(capi.PslError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)
    assert time.perf_counter() - t0 < 20.0
    return str(ei.value)


def test_lookback_wait_gives_up_with_timeout():
    w = inputs.config1()
    dw = engine.upload(w)
    capi.debug_waits(200, capi.DEBUG_LOOKBACK_STALL, 0)
    msg = _expect(capi.PSL_ETIMEOUT, lambda: capi.psl_build(dw.params, dw.records))
    assert "look-back" in msg
    capi.debug_waits(0, 0, 0)
    store = capi.psl_build(dw.params, dw.records)          # the context is still usable
    _, n_valid, _ = store.info()
    assert n_valid == source.psl_build(w.records, w.binning).n_valid


def test_photon_feed_wait_gives_up_with_timeout():
    # enough photons for every warp of the pass to claim a second chunk
    w = inputs.config1(n_histories=2_000_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, 1)
    capi.debug_waits(1000, capi.DEBUG_FEED_STALL, 0)
    msg = _expect(capi.PSL_ETIMEOUT, lambda: capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, w.n_histories))
    assert "incomplete" in msg
    capi.debug_waits(0, 0, 0)
    ref = capi.psl_tally_create(dw.phantom, 1)
    for t in (tally, ref):
        capi.psl_tally_reset(t)
        capi.psl_run(plan, dw.phantom, capi.physics(), t, 0, w.n_histories)
    a, la = engine.raw_tallies(dw, tally, 1)
    b, lb = engine.raw_tallies(dw, ref, 1)
    assert np.array_equal(a, b) and a.sum() > 0 and la[7] == 0


def test_queue_overflow_reports_an_incomplete_tally():
    w = inputs.config1()
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, 1)
    capi.debug_waits(0, 0, 1000)
    msg = _expect(capi.PSL_EOVERFLOW, lambda: capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0,
                                                           w.n_histories))
    assert "overflow" in msg and "incomplete" in msg
    capi.debug_waits(0, 0, 0)
    capi.psl_tally_reset(tally)
    capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, w.n_histories)
    _, lg = engine.raw_tallies(dw, tally, 1)
    assert abs(int(lg[2]) + int(lg[1]) - int(lg[0])) <= 1e-6 * int(lg[0])
