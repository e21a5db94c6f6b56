"""GPU parity of Methods 1 and 2 (Sec. 2.1, 2.2): the phase space read as an
unsorted stream and binned on the fly by type and energy.

Bar: the groups (bin, size, order) and the history order bit-exact against
the oracle's sequential bin fill; the kept particles' weight and energy
bit-exact, positions within 2e-3 cm and directions within 2e-6 of the
oracle's float64 transform; the emitted and missed energy within the
float32-vs-float64 rounding of the per-particle products; the transported
batch gives the same tally, bit for bit, as the same particles given
directly, and balances its energy ledger.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run_both(w, method, first, n, cap):
    """Method `method` on field 0 of w, histories [first, first + n)."""
    dw = engine.upload(w)
    batch = capi.psl_stream_bin(dw.records, w.binning.e_edges, dw.beams[0], method, w.z_psl, w.sad, dw.phantom,
                                first, n, w.seed, cap)
    o = source.stream_bin(w.records, w.binning.e_edges, w.beams[0], method, w.phantom, first, n, cap, w.z_psl, w.sad)
    return dw, batch, o


def _check(batch, o, first):
    ng, n_kept, em, mi = capi.psl_stream_info(batch)
    assert ng == len(o.group_bin)
    nb = int(o.group_count.sum())
    gb = torch.empty(max(ng, 1), dtype=torch.int64, device="cuda")
    gc = torch.empty_like(gb)
    hist = torch.empty(max(nb, 1), dtype=torch.int64, device="cuda")
    capi.psl_stream_read(batch, gb, gc, hist)
    torch.cuda.synchronize()
    assert np.array_equal(gb.cpu().numpy()[:ng], o.group_bin)
    assert np.array_equal(gc.cpu().numpy()[:ng], o.group_count)
    assert np.array_equal(hist.cpu().numpy()[:nb], o.hist)
    # the emitted / missed energy: float32 products on the GPU, float64 here
    assert abs(em - o.emitted) <= 1e-6 * max(o.emitted, 1) + nb
    assert abs(mi - o.missed) <= 1e-6 * max(o.missed, 1) + nb
    # the kept particles: photons first, then charged, each in group order
    _, nph, nel = batch.info()
    assert nph + nel == n_kept
    i = o.hist - first                                   # stream index of each binned particle
    kept = i[o.status[i] == source.ST_TRANSPORT]
    exp = np.r_[kept[o.ptype[kept] == 0], kept[o.ptype[kept] != 0]]
    assert len(exp) == n_kept
    if n_kept:
        st = torch.empty(n_kept * 8, dtype=torch.float32, device="cuda")
        pt = torch.empty(n_kept, dtype=torch.int32, device="cuda")
        pid = torch.empty(n_kept, dtype=torch.int64, device="cuda")
        capi.psl_batch_read(batch, st, pt, pid)
        torch.cuda.synchronize()
        st = st.cpu().numpy().reshape(-1, 8)
        assert np.array_equal(pid.cpu().numpy(), exp + first)
        assert np.array_equal(pt.cpu().numpy(), o.ptype[exp])
        assert np.array_equal(st[:, 7], o.wt[exp])
        assert np.array_equal(st[:, 6], o.e[exp].astype(np.float32))
        assert np.abs(st[:, 0:3] - o.pos[exp]).max() < 2e-3
        assert np.abs(st[:, 3:6] - o.dirs[exp]).max() < 2e-6
    return ng, n_kept


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("n,cap", [(100_000, 4096), (4097, 1), (50_001, 10 ** 9), (1, 3)])
def test_stream_groups_and_particles_bit_exact(method, n, cap):
    w = inputs.config1()
    dw, batch, o = _run_both(w, method, 0, n, cap)
    _check(batch, o, 0)


def test_stream_recycles_and_offsets():
    """A stream longer than the phase space (h reads record h mod N), from a
    non-zero first history, with a fluence map (config 3's)."""
    w = inputs.config3(n_records=200_000)
    n = 450_000
    dw, batch, o = _run_both(w, 2, 123_457, n, 20_000)
    ng, kept = _check(batch, o, 123_457)
    assert kept > 1000 and ng > 10


def test_stream_empty_and_all_rejected():
    w = inputs.config1(n_records=5000)
    dw, batch, o = _run_both(w, 2, 0, 0, 16)
    assert capi.psl_stream_info(batch)[:2] == (0, 0)
    w2 = inputs.config1(n_records=5000)
    b = w2.beams[0]
    b.x1, b.x2 = 30.0, 31.0                      # opening far off the phase space
    dw, batch, o = _run_both(w2, 2, 0, 5000, 16)
    assert len(o.group_bin) == 0
    _check(batch, o, 0)


def test_stream_rejects_bad_arguments():
    w = inputs.config1(n_records=100)
    dw = engine.upload(w)
    for method, cap, n in ((3, 10, 10), (2, 0, 10), (2, 10, -1), (2, 10, 1 << 31)):
        with pytest.raises(capi.PslError):
            capi.psl_stream_bin(dw.records, w.binning.e_edges, dw.beams[0], method, w.z_psl, w.sad, dw.phantom, 0, n,
                                w.seed, cap)


def test_stream_batch_transports_like_its_particles():
    """transport_run of a stream batch = transport of the same particles given
    directly (same ids, same random streams, order-independent integer
    tally), and the ledger balances: deposited + escaped = emitted."""
    w = inputs.config1()
    dw, batch, o = _run_both(w, 2, 0, 60_000, 5000)
    ng, n_kept, em, mi = capi.psl_stream_info(batch)
    st = torch.empty(n_kept * 8, dtype=torch.float32, device="cuda")
    pt = torch.empty(n_kept, dtype=torch.int32, device="cuda")
    pid = torch.empty(n_kept, dtype=torch.int64, device="cuda")
    capi.psl_batch_read(batch, st, pt, pid)
    direct = capi.psl_batch_from_particles(st, pt, pid, w.seed)
    t1 = capi.psl_tally_create(dw.phantom, 1)
    t2 = capi.psl_tally_create(dw.phantom, 1)
    capi.transport_run(dw.phantom, capi.physics(), batch, t1, 0)
    capi.transport_run(dw.phantom, capi.physics(), direct, t2, 0)
    a, la = engine.raw_tallies(dw, t1, 1)
    b, lb = engine.raw_tallies(dw, t2, 1)
    assert np.array_equal(a, b)
    assert la[0] == em and la[1] >= mi
    assert abs(int(la[2]) + int(la[1]) - int(la[0])) <= 1e-6 * int(la[0])
    assert la[2] > 0
