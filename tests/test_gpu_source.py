"""GPU parity of the source stage against the oracle: PSL build (Sec. 2.3.2),
selection and counts (Sec. 2.3.3), reading order, jaw / fluence / MU and the
transform to the phantom surface (Sec. 2.2, 2.3.3, 2.4).

Bar: bit-exact for every integer output (PSL ids, permutation, offsets,
counts, start offsets, entry, read number, record, beam, status) and for the
float32 weight; the rotated / projected float32 state within 2e-5 cm of the
oracle's float64 value (float32 rounding of ~100 cm coordinates).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402
from tests.gpu_util import plan_arrays, source_trace, store_arrays  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _build_both(w):
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    n_records, n_valid, n_bins = store.info()
    ost = source.psl_build(w.records, w.binning)
    return dw, store, ost, n_valid, n_bins


def _check_store(w, store, ost, n_valid, n_bins):
    assert n_valid == ost.n_valid and n_bins == ost.n_bins
    off, perm, rec = store_arrays(store, n_bins, n_valid)
    assert np.array_equal(off, ost.offsets)
    assert np.array_equal(perm, ost.perm)
    r = w.records
    for k, a in enumerate((r.x, r.y, r.u, r.v, r.e, r.wt)):
        assert np.array_equal(rec[:, k], a[ost.perm])            # payload moved bit for bit
    assert np.array_equal(rec[:, 6].view(np.int32), ost.perm.astype(np.int32))
    assert np.array_equal(rec[:, 7].view(np.int32), r.q[ost.perm].astype(np.int32))


@pytest.mark.parametrize("n", [0, 1, 7, 4095, 4096, 4097, 100_003])
def test_build_sizes_and_ragged_tails(n):
    w = inputs.config1(n_records=max(n, 1))
    if n == 0:
        w.records = inputs.Records(*(a[:0] for a in w.records.arrays()))
    dw, store, ost, n_valid, n_bins = _build_both(w)
    _check_store(w, store, ost, n_valid, n_bins)


def test_build_all_records_invalid_and_one_bin():
    w = inputs.config1(n_records=5000)
    w.records.x[:] = 50.0                                     # everything outside the extent
    dw, store, ost, n_valid, n_bins = _build_both(w)
    assert n_valid == 0
    _check_store(w, store, ost, n_valid, n_bins)
    w2 = inputs.config1(n_records=5000)
    w2.binning = inputs.Binning(np.array([-10, 10], np.float32), np.array([-10, 10], np.float32),
                                np.array([0, 10], np.float32), False)
    w2.records.q[:] = 0
    dw, store, ost, n_valid, n_bins = _build_both(w2)
    assert n_bins == 2
    _check_store(w2, store, ost, n_valid, n_bins)


@pytest.mark.parametrize("cfg", [2, 3])
def test_build_full_size(cfg):
    """Full-size phase spaces (1e7 records, 9216 PSLs; 4e7 records, 102,400 PSLs)."""
    w = inputs.config2(n_histories=1000) if cfg == 2 else inputs.config3(n_histories=1000)
    dw, store, ost, n_valid, n_bins = _build_both(w)
    _check_store(w, store, ost, n_valid, n_bins)


def _plan_both(w, store, ost, n_sim=None):
    n_sim = w.n_histories if n_sim is None else n_sim
    dw = engine.upload(w)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, n_sim, w.seed)
    opl = source.make_plan(ost, w.beams, n_sim, w.seed, w.z_psl, w.sad)
    (beam, psl, count, offset), n_total = plan_arrays(plan)
    assert n_total == opl.n_total_psl
    assert np.array_equal(beam, opl.field) and np.array_equal(psl, opl.psl)
    assert np.array_equal(count, opl.count) and np.array_equal(offset, opl.offset)
    return dw, plan, opl


def _check_trace(w, dw, plan, store_o, opl, hs):
    h0, n = int(hs[0]), len(hs)
    g = source_trace(dw, plan, h0, n)
    o = source.source(opl, store_o, w.records, w.beams, w.phantom, hs, w.z_psl, w.sad)
    assert np.array_equal(g["entry"], o.entry) and np.array_equal(g["use"], o.use)
    assert np.array_equal(g["rec"], o.rec) and np.array_equal(g["beam"], o.beam)
    assert np.array_equal(g["status"], o.status)
    ok = o.status == source.ST_TRANSPORT
    assert np.array_equal(g["ptype"][ok], o.ptype[ok])
    assert np.array_equal(g["state"][ok, 7], o.wt[ok])                       # weight bit-exact
    assert np.array_equal(g["state"][ok, 6], o.e[ok].astype(np.float32))
    assert np.abs(g["state"][ok, 0:3] - o.pos[ok]).max() < 2e-5 * 100
    assert np.abs(g["state"][ok, 3:6] - o.dir[ok]).max() < 2e-6
    return ok.sum()


def test_source_config1_all_histories():
    w = inputs.config1()
    dw, store, ost, n_valid, n_bins = _build_both(w)
    dw, plan, opl = _plan_both(w, store, ost)
    n_ok = int(_check_trace(w, dw, plan, ost, opl, np.arange(w.n_histories)))
    assert n_ok > 0.3 * w.n_histories, n_ok


def test_source_multibeam_fluence_rotations():
    """Config-4 style plan on a small phase space: 200+ segments, gantry angles,
    fluence maps and MU weights."""
    w = inputs.config4(n_records=200_000, n_histories=300_000)
    dw, store, ost, n_valid, n_bins = _build_both(w)
    dw, plan, opl = _plan_both(w, store, ost)
    assert int(_check_trace(w, dw, plan, ost, opl, np.arange(100_000, 160_000))) > 1000


@pytest.mark.parametrize("cfg", [2, 3])
def test_source_full_size_sampled(cfg):
    """Full-size plans (1e8 / 1e9 histories): the integer plan is compared
    whole; the source stage on sampled ranges spread over all groups."""
    w = inputs.config2() if cfg == 2 else inputs.config3()
    dw, store, ost, n_valid, n_bins = _build_both(w)
    dw, plan, opl = _plan_both(w, store, ost)
    rng = np.random.default_rng(cfg)
    for h0 in list(rng.integers(0, w.n_histories - 64, 12)) + [0, w.n_histories - 64]:
        hs = np.arange(h0, h0 + 64)
        g = source_trace(dw, plan, int(h0), 64)
        ent, use = source.history_map(opl, hs, literal_limit=0)
        assert np.array_equal(g["entry"], ent) and np.array_equal(g["use"], use)
        rec = opl.start[ent] + (opl.offset[ent] + use) % opl.nrec[ent]
        assert np.array_equal(g["rec"], rec)


def test_source_strided_batches():
    """Independent batches: batch b reads histories b, b + N_b, ... (bit-exact)."""
    w = inputs.config1()
    dw, store, ost, n_valid, n_bins = _build_both(w)
    dw, plan, opl = _plan_both(w, store, ost)
    for b in (0, 3, 9):
        hs = np.arange(b, w.n_histories, 10)
        g = source_trace(dw, plan, b, len(hs), stride=10)
        o = source.source(opl, ost, w.records, w.beams, w.phantom, hs, w.z_psl, w.sad)
        assert np.array_equal(g["rec"], o.rec) and np.array_equal(g["status"], o.status)
        ok = o.status == source.ST_TRANSPORT
        assert np.array_equal(g["state"][ok, 7], o.wt[ok])
    # every energy division appears in every batch
    for b in (0, 9):
        ent, _ = source.history_map(opl, np.arange(b, w.n_histories, 10))
        assert set(np.unique(opl.group[ent])) == set(np.unique(opl.group[opl.count > 0]))


# ---------------------------------------------------- redistribution (APR) ---
def _apr_workload(w, k, seed):
    w.binning.apr_copies, w.binning.apr_seed = k, seed
    return dataclasses.replace(w, records=source.apr_expand(w.records, k, seed))


@pytest.mark.parametrize("k,n", [(2, 4097), (4, 100_000), (7, 1), (3, 0)])
def test_apr_store_bit_exact(k, n):
    """psl_build with K copies per record (Sec. 2.3.1): the rotated records,
    their PSL ids, order and offsets equal the oracle's bit for bit."""
    w = inputs.config1(n_records=max(n, 1))
    if n == 0:
        w.records = inputs.Records(*(a[:0] for a in w.records.arrays()))
    we = _apr_workload(w, k, 0xA5A5000012340000 + k)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    n_records, n_valid, n_bins = store.info()
    assert n_records == k * n
    ost = source.psl_build(we.records, w.binning)
    _check_store(we, store, ost, n_valid, n_bins)


def test_apr_full_size_store():
    """The 1e7-record phase space with 3 copies (3e7 sorted records)."""
    w = inputs.config2(n_histories=1000)
    we = _apr_workload(w, 3, 0x5EED)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    n_records, n_valid, n_bins = store.info()
    assert n_records == 3 * w.records.n
    _check_store(we, store, source.psl_build(we.records, w.binning), n_valid, n_bins)


def test_apr_source_stage_bit_exact():
    """Plan and source stage over a redistributed store, every history."""
    w = inputs.config1()
    we = _apr_workload(w, 4, 99)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    ost = source.psl_build(we.records, w.binning)
    dw, plan, opl = _plan_both(we, store, ost)
    n_ok = int(_check_trace(we, dw, plan, ost, opl, np.arange(w.n_histories)))
    assert n_ok > 0.3 * w.n_histories, n_ok


def test_apr_rejects_bad_copy_counts():
    w = inputs.config1(n_records=100)
    for k in (0, -2, 1 << 24):
        w.binning.apr_copies = k
        dw = engine.upload(w)
        with pytest.raises(capi.PslError):
            capi.psl_build(dw.params, dw.records)
    w.binning.apr_copies = 2
    dw = engine.upload(w)
    nb = w.binning.n_bins
    off = torch.empty(nb + 1, dtype=torch.int64, device="cuda")
    rec = torch.empty(100 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.PslError):                 # the allocation-free build takes no copies
        capi.psl_build_static(dw.params, dw.records, off, rec)


def test_plan_beyond_2_32_histories():
    """A 6e9-history plan (the size that reaches 1 % at the isocentre): the
    integer plan whole, and the source stage on ranges past 2^32, bit-exact."""
    w = inputs.config2(n_histories=6_000_000_000)
    dw, store, ost, n_valid, n_bins = _build_both(w)
    dw, plan, opl = _plan_both(w, store, ost)
    for h0 in (0, (1 << 32) - 32, 5_123_456_789, w.n_histories - 64):
        hs = np.arange(h0, h0 + 64)
        g = source_trace(dw, plan, int(h0), 64)
        ent, use = source.history_map(opl, hs, literal_limit=0)
        assert np.array_equal(g["entry"], ent) and np.array_equal(g["use"], use)
        rec = opl.start[ent] + (opl.offset[ent] + use) % opl.nrec[ent]
        assert np.array_equal(g["rec"], rec)
    with pytest.raises(capi.PslError):              # some PSL would get >= 2^32 histories
        capi.psl_plan_create(store, dw.beams, w.sad, 1 << 61, w.seed)
