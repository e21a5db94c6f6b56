"""Pins of the oracle of Methods 1 and 2 (Sec. 2.1, 2.2): the phase space as
an unsorted stream, binned on the fly by type and energy.

The bin-fill procedure is pinned by a hand-worked trace and by its closed
characterisation (every binned particle exactly once; groups homogeneous;
a bin's full groups are its particles ranked [jC, (j+1)C) in stream order,
sent when the last of them arrives; the rest sent at the end in bin order);
the source side by the point-source jaw closed form and by recycling.
"""
import numpy as np
import pytest

from oracle import _lib, source
from paper_1302_1861_b300 import inputs


def _bin(key, nbins, cap):
    key = np.ascontiguousarray(key, np.int32)
    n = len(key)
    gb, gc, order = (np.zeros(max(n, 1), np.int64) for _ in range(3))
    ng = _lib.lib().ora_stream_bin(n, _lib._p(key), nbins, cap, _lib._p(gb), _lib._p(gc), _lib._p(order))
    assert ng >= 0
    return gb[:ng], gc[:ng], order[:int(gc[:ng].sum())]


def test_hand_worked_stream():
    # capacity 2, bins 0..2, -1 = rejected.  By hand: bin 0 fills at i=2 ->
    # (0: 0, 2); bin 1 at i=5 -> (1: 1, 5); bin 0 at i=7 -> (0: 4, 7); bin 1
    # at i=9 -> (1: 8, 9); end of stream: bin 2 holds 6 -> (2: 6).
    key = [0, 1, 0, -1, 0, 1, 2, 0, 1, 1]
    gb, gc, order = _bin(key, 3, 2)
    assert gb.tolist() == [0, 1, 0, 1, 2]
    assert gc.tolist() == [2, 2, 2, 2, 1]
    assert order.tolist() == [0, 2, 1, 5, 4, 7, 8, 9, 6]


def _characterisation(key, nbins, cap):
    """The groups in the closed form: per bin b, its particles in stream
    order p_b[0..c_b); full group j = p_b[jC..(j+1)C), sent at p_b[(j+1)C-1];
    then the partial remainders in bin order."""
    key = np.asarray(key)
    full, part = [], []
    for b in range(nbins):
        pb = np.flatnonzero(key == b)
        nf = len(pb) // cap
        for j in range(nf):
            full.append((pb[(j + 1) * cap - 1], b, pb[j * cap:(j + 1) * cap]))
        if len(pb) % cap:
            part.append((b, pb[nf * cap:]))
    full.sort(key=lambda t: t[0])
    gb = [b for _, b, _ in full] + [b for b, _ in part]
    gc = [len(m) for _, _, m in full] + [len(m) for _, m in part]
    order = [int(i) for _, _, m in full for i in m] + [int(i) for _, m in part for i in m]
    return gb, gc, order


@pytest.mark.parametrize("n,nbins,cap,seed", [(1, 4, 1, 0), (1000, 8, 7, 1), (5000, 64, 33, 2), (3000, 6, 1, 3),
                                              (2000, 10, 100000, 4), (4097, 2, 4096, 5), (0, 4, 3, 6)])
def test_closed_form_of_the_bin_fill(n, nbins, cap, seed):
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(np.ones(nbins + 1))          # uneven bin populations, -1 last
    key = rng.choice(np.r_[np.arange(nbins), -1], size=n, p=p).astype(np.int32)
    gb, gc, order = _bin(key, nbins, cap)
    egb, egc, eorder = _characterisation(key, nbins, cap)
    assert gb.tolist() == egb and gc.tolist() == egc and order.tolist() == eorder
    # every binned particle exactly once, every group homogeneous and <= capacity
    assert sorted(order.tolist()) == np.flatnonzero(key >= 0).tolist()
    starts = np.r_[0, np.cumsum(gc)]
    for g in range(len(gb)):
        assert np.all(key[order[starts[g]:starts[g + 1]]] == gb[g]) and 1 <= gc[g] <= cap


def test_large_capacity_is_a_stable_sort_and_unit_capacity_the_stream():
    rng = np.random.default_rng(9)
    key = rng.integers(-1, 12, 3000).astype(np.int32)
    gb, gc, order = _bin(key, 12, 10 ** 9)
    keep = np.flatnonzero(key >= 0)
    assert order.tolist() == keep[np.argsort(key[keep], kind="stable")].tolist()
    gb1, gc1, order1 = _bin(key, 12, 1)
    assert order1.tolist() == keep.tolist() and np.all(gc1 == 1) and np.array_equal(gb1, key[keep])


def _open_field(w, size):
    b = w.beams[0]
    b.x1, b.x2, b.y1, b.y2 = -size / 2, size / 2, -size / 2, size / 2
    b.fluence = None
    return b


def test_method2_point_source_jaw_closed_form():
    """Records from a point source at the origin: a straight line through the
    jaw planes is inside the opening exactly when its position scaled to SAD
    is inside the field (away from the edges, where float32 rounding decides)."""
    w = inputs.config1(n_records=40000)
    beam = _open_field(w, 4.0)
    r = w.records
    # the config-1 records point back at the source: u = x / |(x, y, z_psl)|
    out = source.stream_bin(r, w.binning.e_edges, beam, source.METHOD_JAW_MODEL, w.phantom, 0, r.n, 1000,
                            w.z_psl, w.sad)
    xs, ys = r.x.astype(np.float64) * w.sad / w.z_psl, r.y.astype(np.float64) * w.sad / w.z_psl
    inside = (np.abs(xs) < 2.0 - 1e-4) & (np.abs(ys) < 2.0 - 1e-4)
    outside = (np.abs(xs) > 2.0 + 1e-4) | (np.abs(ys) > 2.0 + 1e-4)
    passed = (out.status == source.ST_TRANSPORT) | (out.status == source.ST_MISS)
    assert np.all(passed[inside]) and not np.any(passed[outside])
    # method 1 takes every record, with its own weight
    out1 = source.stream_bin(r, w.binning.e_edges, beam, source.METHOD_PATIENT_DEPENDENT, w.phantom, 0, r.n, 1000,
                             w.z_psl, w.sad)
    ok1 = (out1.status == source.ST_TRANSPORT) | (out1.status == source.ST_MISS)
    assert ok1.all() and np.array_equal(out1.wt, r.wt)
    assert set(out.hist.tolist()) <= set(out1.hist.tolist())


def test_stream_recycling_and_bins():
    w = inputs.config1(n_records=3000)
    beam = _open_field(w, 6.0)
    ee = w.binning.e_edges
    n = int(2.5 * w.records.n)
    out = source.stream_bin(w.records, ee, beam, source.METHOD_JAW_MODEL, w.phantom, 100, n, 50, w.z_psl, w.sad)
    N = w.records.n
    # history h reads record h mod N: histories N apart agree
    assert np.array_equal(out.status[:n - N], out.status[N:])
    assert np.array_equal(out.key[:n - N], out.key[N:])
    # bins: type major, energy bin by the interior edges
    h = out.hist - 100
    e = out.e[h]
    q = w.records.q[(out.hist) % N]
    ne = len(ee) - 1
    eb = np.searchsorted(ee[1:-1], e.astype(np.float32), side="right")
    assert np.array_equal(out.key[h], (q != 0) * ne + eb)
    # the emitted energy is that of the binned particles, the missed part of it
    fp = np.rint(out.e * out.wt.astype(np.float64) * 2.0 ** 32).astype(np.int64)
    assert out.emitted == int(fp[h].sum())
    assert out.missed == int(fp[h][out.status[h] == source.ST_MISS].sum())
