"""Pins of the oracle's random numbers and source stage (CPU only).

Each test checks the oracle against something other than itself: published
known-answer vectors, brute force on tiny inputs, closed geometric cases and
exact integer identities of the count equations of Sec. 2.3.3.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import source
from paper_1302_1861_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ---
def test_philox_known_answers():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(t, 16) for t in line.split()])
    rows = np.array(rows, np.uint64)
    out = oracle.philox(rows[:, 0:4].astype(np.uint32), rows[:, 4:6].astype(np.uint32))
    assert np.array_equal(out.astype(np.uint64), rows[:, 6:10])


def test_uniform_is_exact_midpoint_grid():
    # the uniform of a draw is ((r >> 9) + 0.5) 2^-23: strictly inside (0, 1)
    # and exactly representable in float32 (24 significant bits)
    r = oracle.philox(np.arange(4000, dtype=np.uint32).reshape(-1, 4), np.array([1, 2], np.uint32)).ravel()
    u = ((r >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    assert (u > 0).all() and (u < 1).all()
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    # roughly uniform: mean and variance of 16000 draws
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


# -------------------------------------------------------- PSL generation ---
def _tiny_records(n=300, seed=5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-3.5, 3.5, n).astype(np.float32)
    y = rng.uniform(-3.5, 3.5, n).astype(np.float32)
    x[:5] = [-3.0, 3.0, 0.0, 1.0, -1.0]       # values on bin edges
    e = rng.uniform(-0.1, 6.5, n).astype(np.float32)
    e[5:9] = [0.6, 6.0, 0.0, 1.2]              # on energy edges, top edge, zero
    q = rng.choice(np.array([0, 0, 0, -1, 1], np.int8), n)
    z = np.zeros(n, np.float32)
    return inputs.Records(x, y, z, z, e, np.ones(n, np.float32), q)


def _brute_key(x, y, e, q, xe, ye, ee):
    nx, ny, ne = len(xe) - 1, len(ye) - 1, len(ee) - 1
    bx = [i for i in range(nx) if xe[i] <= x < xe[i + 1]]
    by = [j for j in range(ny) if ye[j] <= y < ye[j + 1]]
    if not bx or not by or not (e > 0):
        return 2 * ne * nx * ny
    # energy: bins between interior edges, open at both ends
    eb = sum(1 for k in range(1, ne) if ee[k] <= e)
    t = 0 if q == 0 else 1
    return (t * ne + eb) * nx * ny + by[0] * nx + bx[0]


@pytest.mark.parametrize("log_ebins", [False, True])
def test_psl_build_matches_brute_force(log_ebins):
    rec = _tiny_records()
    b = inputs.make_binning(3.0, 1.0, 10 if not log_ebins else 32, log_ebins)
    st = source.psl_build(rec, b)
    keys = [_brute_key(float(rec.x[i]), float(rec.y[i]), float(rec.e[i]), int(rec.q[i]),
                       b.x_edges.astype(float), b.y_edges.astype(float), b.e_edges.astype(float))
            for i in range(rec.n)]
    assert list(st.keys) == keys
    # stable sort by key: Python's sorted on (key, index) pairs, invalid dropped
    expect = [i for k, i in sorted((k, i) for i, k in enumerate(keys)) if k < b.n_bins]
    assert list(st.perm) == expect
    counts = np.zeros(b.n_bins, np.int64)
    for k in keys:
        if k < b.n_bins:
            counts[k] += 1
    assert st.offsets[0] == 0
    assert np.array_equal(np.diff(st.offsets), counts)


def test_psl_build_invariants_config1():
    w = inputs.config1(n_records=20000)
    st = source.psl_build(w.records, w.binning)
    k = st.keys[st.perm]
    assert (np.diff(k) >= 0).all()                      # sorted
    assert len(np.unique(st.perm)) == len(st.perm)      # a permutation of the valid records
    same = np.diff(k) == 0
    assert (np.diff(st.perm)[same] > 0).all()            # stable: equal keys keep input order
    # Gaussian tails outside the [-3, 3) cm extent are the only dropped records
    x, y = w.records.x, w.records.y
    inside = (x >= -3) & (x < 3) & (y >= -3) & (y < 3)
    assert st.n_valid == int(inside.sum()) < w.records.n


# -------------------------------------------------------------- selection ---
def test_roi_selection_matches_overlap_area():
    b = inputs.make_binning(20.0, 1.0, 4, True)
    for beam in (inputs.Beam(-5, 5, -5, 5), inputs.Beam(-2.5, 7.25, -15, 1.0, roi_margin=0.5),
                 inputs.Beam(-2, 2, -2, 2, roi_margin=0.0)):
        sel = source.roi_select(b.x_edges, b.y_edges, beam, 100.0, 100.0)
        xe, ye = b.x_edges.astype(np.float32), b.y_edges.astype(np.float32)
        m = np.float32(beam.roi_margin)
        rx = (np.float32(beam.x1) - m, np.float32(beam.x2) + m)
        ry = (np.float32(beam.y1) - m, np.float32(beam.y2) + m)
        for j in range(len(ye) - 1):
            for i in range(len(xe) - 1):
                wx = min(xe[i + 1], rx[1]) - max(xe[i], rx[0])
                wy = min(ye[j + 1], ry[1]) - max(ye[j], ry[0])
                assert sel[j, i] == (wx > 0 and wy > 0)
    # a 4x4 field with no margin selects exactly 4x4 positions (touching edges excluded)
    sel = source.roi_select(b.x_edges, b.y_edges, inputs.Beam(-2, 2, -2, 2, roi_margin=0.0), 100.0, 100.0)
    assert sel.sum() == 16


def test_roi_back_projection_scales_with_plane():
    # PSL plane at half the SAD: the ROI halves (Fig. 1 back-projection)
    b = inputs.make_binning(10.0, 0.5, 2, False)
    s1 = source.roi_select(b.x_edges, b.y_edges, inputs.Beam(-4, 4, -4, 4, roi_margin=0.0), 50.0, 100.0)
    assert s1.sum() == 64   # +-2 cm at the plane: 8 x 8 bins of 0.5 cm
    s2 = source.roi_select(b.x_edges, b.y_edges, inputs.Beam(-4, 4, -4, 4, roi_margin=0.0), 100.0, 100.0)
    assert s2.sum() == 256  # +-4 cm at SAD itself


def _plan_for(w, n_sim):
    st = source.psl_build(w.records, w.binning)
    return st, source.make_plan(st, w.beams, n_sim, w.seed, w.z_psl, w.sad)


@pytest.mark.parametrize("n_sim", [1, 977, 100_000, 10 ** 9 + 7])
def test_counts_sum_and_share(n_sim):
    w = inputs.config1(n_records=5000)
    w.beams = [inputs.Beam(-2, 2, -2, 2, mu=1.0), inputs.Beam(-1, 2.5, -3, 0.5, mu=2.0)]
    st, pl = _plan_for(w, n_sim)
    assert int(pl.count.sum()) == n_sim                                   # sum_ij N_ij = N_sim
    assert pl.n_total_psl == int(pl.nrec.sum())                           # N_total^psl = sum_i sum_j N_j
    share = n_sim * pl.nrec.astype(float) / pl.n_total_psl
    assert (np.abs(pl.count - share) < 1.0 + 1e-9 * share).all()         # |N_ij - share| < 1
    assert (pl.count[pl.nrec == 0] == 0).all()


def test_reading_order_is_round_robin():
    """Literal round-robin (Sec. 2.3.3): energy division outermost, photons
    then electrons, then rounds of one read per PSL still owed histories."""
    w = inputs.config1(n_records=3000)
    st, pl = _plan_for(w, 2500)
    expect = []
    for e in range(pl.n_ebins):
        for t in (0, 1):
            g = 2 * e + t
            ents = [k for k in range(len(pl.count)) if pl.group[k] == g and pl.count[k] > 0]
            ents.sort(key=lambda k: (-int(pl.count[k]), k))
            r = 0
            while True:
                active = [k for k in ents if pl.count[k] > r]
                if not active:
                    break
                expect += [(k, r) for k in active]
                r += 1
    ent, use = source.history_map(pl, np.arange(2500))
    assert list(zip(ent.tolist(), use.tolist())) == expect
    # the per-history lookup (used for sampled histories) agrees with it
    hs = np.array([0, 1, 17, 999, 1500, 2499])
    e2, u2 = source.history_map(pl, hs, literal_limit=0)
    assert np.array_equal(e2, ent[hs]) and np.array_equal(u2, use[hs])


def test_random_start_and_wrap():
    w = inputs.config1(n_records=400)
    st, pl = _plan_for(w, 50_000)        # far more histories than records: recycling
    h = np.arange(50_000)
    ent, use = source.history_map(pl, h)
    rec = pl.start[ent] + (pl.offset[ent] + use) % pl.nrec[ent]
    assert ((rec >= pl.start[ent]) & (rec < pl.start[ent] + pl.nrec[ent])).all()
    # each entry reads its PSL cyclically from its random start
    k = int(np.argmax(pl.count))
    r = rec[ent == k]
    assert r[0] == pl.start[k] + pl.offset[k]
    assert np.array_equal(np.diff(r) % pl.nrec[k], np.ones(len(r) - 1) % pl.nrec[k])
    # random starts spread uniformly over the PSLs' records
    st2, pl2 = _plan_for(inputs.config1(n_records=50000), 1000)
    big = pl2.nrec >= 50
    offs = (pl2.offset[big] + 0.5) / pl2.nrec[big]
    assert big.sum() > 100 and 0.4 < offs.mean() < 0.6 and (pl2.offset < np.maximum(pl2.nrec, 1)).all()


# ------------------------------------------------------- source transform ---
def _point_source_workload(jaws, n=20000):
    w = inputs.config1(n_records=n, n_histories=n)
    w.beams = [inputs.Beam(*jaws, roi_margin=2.0)]
    return w


def test_jaw_model_equals_field_at_sad_for_point_source():
    """Straight rays from a point source: the jaw test at any jaw plane keeps
    the same particles as the field rectangle at SAD (Sec. 2.2)."""
    w = _point_source_workload((-1.5, 2.0, -2.0, 1.0))
    st, pl = _plan_for(w, w.n_histories)
    s = source.source(pl, st, w.records, w.beams, w.phantom, np.arange(w.n_histories), w.z_psl, w.sad)
    src = st.perm[s.rec]
    xs = w.records.x[src].astype(float) * w.sad / w.z_psl
    ys = w.records.y[src].astype(float) * w.sad / w.z_psl
    b = w.beams[0]
    inside = (xs >= b.x1) & (xs <= b.x2) & (ys >= b.y1) & (ys <= b.y2)
    acc = s.status != source.ST_JAW
    tol = 1e-4
    near = (np.minimum.reduce([np.abs(xs - b.x1), np.abs(xs - b.x2), np.abs(ys - b.y1), np.abs(ys - b.y2)]) < tol)
    assert np.array_equal(acc[~near], inside[~near])
    assert acc.sum() > 1000


def test_unit_fluence_and_single_beam_keep_weights():
    w = _point_source_workload((-2, 2, -2, 2))
    w.beams[0].fluence = np.ones((40, 40), np.float32)
    w.beams[0].mu = 3.7
    st, pl = _plan_for(w, w.n_histories)
    s = source.source(pl, st, w.records, w.beams, w.phantom, np.arange(5000), w.z_psl, w.sad)
    ok = s.status == source.ST_TRANSPORT
    assert np.array_equal(s.wt[ok], w.records.wt[st.perm[s.rec[ok]]])


def test_mu_weights_and_fluence_lookup():
    w = _point_source_workload((-3, 3, -3, 3))
    f = np.arange(1600, dtype=np.float32).reshape(40, 40) / 1600
    w.beams = [inputs.Beam(-3, 3, -3, 3, mu=1.0, fluence=f), inputs.Beam(-3, 3, -3, 3, mu=3.0)]
    st, pl = _plan_for(w, w.n_histories)
    s = source.source(pl, st, w.records, w.beams, w.phantom, np.arange(8000), w.z_psl, w.sad)
    ok = s.status == source.ST_TRANSPORT
    src = st.perm[s.rec]
    # PSL plane = iso plane: no projection; cell = floor(x + 20) in float32
    xi, yi = w.records.x[src], w.records.y[src]
    b0 = ok & (s.beam == 0)
    ix = np.floor(xi[b0] + np.float32(20)).astype(int)
    iy = np.floor(yi[b0] + np.float32(20)).astype(int)
    exp0 = f[iy, ix] * 0.25
    assert np.allclose(s.wt[b0], exp0, rtol=1e-6, atol=1e-7)
    b1 = ok & (s.beam == 1)
    assert np.allclose(s.wt[b1], 0.75, rtol=1e-7)


# (destination axis, sign) of input axes x, y, z under a gantry rotation
# about +y: x -> z sin g ..., i.e. (x, y, z) -> (x cos g + z sin g, y, z cos g - x sin g)
@pytest.mark.parametrize("gantry,perm", [(0.0, ((0, 1), (1, 1), (2, 1))),
                                          (90.0, ((2, -1), (1, 1), (0, 1))),
                                          (180.0, ((0, -1), (1, 1), (2, -1))),
                                          (270.0, ((2, 1), (1, 1), (0, -1)))])
def test_gantry_rotations_are_exact_permutations(gantry, perm):
    R = source.beam_matrix(inputs.Beam(-1, 1, -1, 1, gantry=gantry))
    d = np.array([0.3, -0.2, 0.9])
    out = R @ d
    expect = np.zeros(3)
    for j, (src, sgn) in enumerate(perm):
        expect[src] = sgn * d[j]
    assert np.array_equal(out, expect)


def test_rotation_order_collimator_then_gantry():
    b = inputs.Beam(-1, 1, -1, 1, gantry=90.0, collimator=90.0)
    R = source.beam_matrix(b)
    # collimator 90 maps x->y; gantry 90 then leaves y unchanged
    assert np.array_equal(R @ np.array([1.0, 0, 0]), np.array([0, 1.0, 0]))
    assert np.array_equal(R @ np.array([0, 0, 1.0]), np.array([1.0, 0, 0]))


def test_projection_to_phantom_surface():
    w = _point_source_workload((-2, 2, -2, 2))
    st, pl = _plan_for(w, w.n_histories)
    s = source.source(pl, st, w.records, w.beams, w.phantom, np.arange(3000), w.z_psl, w.sad)
    ok = s.status == source.ST_TRANSPORT
    # gantry 0: every particle enters through the top face z = 0 (SSD 90)
    assert np.allclose(s.pos[ok, 2], 0.0, atol=1e-9)
    # and lies on its straight line from the point source
    src = st.perm[s.rec[ok]]
    x_expect = w.records.x[src].astype(float) * 90.0 / 100.0 + 8.0
    assert np.allclose(s.pos[ok, 0], x_expect, atol=2e-5)
    # energy ledger: emitted is the fixed-point sum of E*wt of accepted histories
    fp = np.rint(s.e[ok] * s.wt[ok].astype(float) * 2.0 ** 32).astype(np.int64).sum()
    assert fp + s.missed_fp == s.emitted_fp
