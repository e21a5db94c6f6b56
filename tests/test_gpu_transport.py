"""GPU parity of transport, tally and readout against the oracle
(Sec. 2.3.3 dose counters and batches, Sec. 2.5 normalisation).

Bars (FP32 transport against the FP64 oracle on the same Philox streams):
* closed forms: narrow-beam attenuation exp(-mu x) and channel fractions
  within 5 binomial standard deviations; CSDA path of a straight electron
  within 1e-4 relative; energy ledger deposited + escaped = emitted within
  1e-6 relative;
* event level: per-history deposited energy equal to the oracle's within
  1e-4 relative for >= 97 % of histories (the rest are histories in which an
  FP32/FP64 rounding difference flipped a branch: they must still conserve
  energy);
* dose (config 1, 1e5 histories): mean relative difference < 0.5 % over
  voxels above 10 % of the maximum, >= 99 % of them within 3 combined
  standard deviations, gamma 2 %/2 mm >= 99 %.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import _lib, readout, source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402
from tests.gpu_util import transport_particles  # noqa: E402

FP = 2.0 ** 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _column_workload(nz, vz, rho=None, mat=None, nxy=1, vxy=1.0):
    w = inputs.config1(n_records=100, n_histories=100)
    m = np.zeros((nz, nxy, nxy), np.uint8) if mat is None else mat
    r = np.ones((nz, nxy, nxy), np.float32) if rho is None else rho
    w.phantom = inputs.Phantom(m, r, (vxy, vxy, vz), (0.0, 0.0, 0.0))
    return w


def _pencil(n, ptype, E, x=0.5, y=0.5):
    return (np.full(n, ptype, np.int32), np.tile([x, y, 0.0], (n, 1)), np.tile([0.0, 0.0, 1.0], (n, 1)),
            np.full(n, E), np.ones(n), np.arange(n, dtype=np.uint64))


@pytest.mark.parametrize("E", [0.1, 1.0, 6.0])
def test_narrow_beam_attenuation(E):
    w = _column_workload(40, 1.0)
    dw = engine.upload(w)
    n = 400_000
    t, lg = transport_particles(dw, *_pencil(n, 0, E), seed=21, flags=capi.PHYS_FIRST_INTERACTION)
    mu = _lib.lib().ora_mu_rho(E, 0, 3)
    beyond = n - np.cumsum(t[:, 0, 0] / (np.float32(E) * FP))
    p = np.exp(-mu * np.arange(1, 41))
    sd = np.sqrt(n * p * (1 - p)) + 1
    assert (np.abs(beyond - n * p) < 5 * sd).all()


@pytest.mark.parametrize("E,mat", [(0.04, 0), (0.04, 1), (6.0, 0), (3.0, 1)])
def test_channel_fractions(E, mat):
    w = _column_workload(20, 1.0, mat=np.full((20, 1, 1), mat, np.uint8))
    dw = engine.upload(w)
    n = 400_000
    _, lg = transport_particles(dw, *_pencil(n, 0, E), seed=22, flags=capi.PHYS_FIRST_INTERACTION)
    k = lg[3:6].astype(float)
    mus = np.array([_lib.lib().ora_mu_rho(E, mat, c) for c in range(3)])
    p = mus / mus.sum()
    sd = np.sqrt(k.sum() * p * (1 - p)) + 1
    assert (np.abs(k - k.sum() * p) < 5 * sd).all()


@pytest.mark.parametrize("T0,rho", [(2.0, 1.0), (0.9, 0.26), (5.0, 1.85)])
def test_csda_range_and_track(T0, rho):
    """Straight electron, no hard events: the dose profile ends where the
    oracle's does (both follow the CSDA range), all on the track."""
    nz = 200
    w = _column_workload(nz, 0.05, rho=np.full((nz, 1, 1), rho, np.float32))
    dw = engine.upload(w)
    n = 8
    flags = capi.PHYS_NO_MSC | capi.PHYS_NO_HARD | capi.PHYS_LOCAL_SECONDARIES
    t, lg = transport_particles(dw, *_pencil(n, 1, T0), seed=3, flags=flags)
    to, lo, ho = oracle.transport(*_pencil(n, 1, T0), w.phantom, seed=3, flags=flags, per_history=True)
    csda = ho["path"][0]
    last = int(math.floor(csda / 0.05))
    prof = t[:, 0, 0].astype(float)
    assert prof[last + 2:].sum() == 0 and (prof[: last - 1] > 0).all()
    # energy per voxel along the track agrees with the oracle to 1e-4 (relative to the total)
    assert np.abs(prof - to[:, 0, 0]).sum() < 1e-4 * prof.sum() + 4
    assert abs(int(lg[2]) - n * np.float32(T0) * FP) < 1e-6 * n * T0 * FP


@pytest.mark.parametrize("T0,rho", [(2.0, 1.0), (5.0, 1.85)])
def test_csda_range_and_track_positron(T0, rho):
    """Straight positron, no hard events: its own (Bhabha) range table; the
    dose profile follows the oracle's, and the 2 m c^2 of the annihilation
    at rest is deposited where it stops (secondaries local)."""
    nz = 200
    w = _column_workload(nz, 0.05, rho=np.full((nz, 1, 1), rho, np.float32))
    dw = engine.upload(w)
    n = 8
    flags = capi.PHYS_NO_MSC | capi.PHYS_NO_HARD | capi.PHYS_LOCAL_SECONDARIES
    t, lg = transport_particles(dw, *_pencil(n, 2, T0), seed=3, flags=flags)
    to, lo, ho = oracle.transport(*_pencil(n, 2, T0), w.phantom, seed=3, flags=flags, per_history=True)
    prof = t[:, 0, 0].astype(float)
    assert np.abs(prof - to[:, 0, 0]).sum() < 1e-4 * prof.sum() + 4
    e_all = n * (np.float32(T0) + 2 * np.float32(oracle.ME)) * FP
    assert abs(int(lg[2]) - e_all) < 1e-6 * e_all


@pytest.mark.parametrize("ptype", [1, 2])
def test_hard_collision_counts_match_oracle(ptype):
    """Hard Moller (electrons) and Bhabha (positrons) collisions of 3 MeV
    particles crossing 0.5 mm of water on the same random streams: the
    GPU's count (ledger slot 11) equals the oracle's up to the rare
    histories a float32 rounding flips, and the two species differ."""
    w = _column_workload(1, 0.05)
    dw = engine.upload(w)
    n = 400_000
    phys_flags = capi.PHYS_NO_MSC | capi.PHYS_LOCAL_SECONDARIES
    # W_cb above the energy: no hard bremsstrahlung
    st = np.concatenate([np.tile([0.5, 0.5, 0.0, 0.0, 0.0, 1.0], (n, 1)), np.full((n, 1), 3.0), np.ones((n, 1))],
                        1).astype(np.float32)
    batch = capi.psl_batch_from_particles(torch.from_numpy(st).cuda(),
                                          torch.full((n,), ptype, dtype=torch.int32).cuda(),
                                          torch.arange(n, dtype=torch.int64).cuda(), 8)
    tally = capi.psl_tally_create(dw.phantom, 1)
    capi.transport_run(dw.phantom, capi.physics(phys_flags, wcb=10.0), batch, tally, 0)
    _, lg = engine.raw_tallies(dw, tally, 1)
    _, lo = oracle.transport(*_pencil(n, ptype, 3.0), w.phantom, seed=8, flags=phys_flags, wcb=10.0)
    g, o = int(lg[11]), int(lo[oracle.L_HARD_COLL])
    assert o > 5000
    assert abs(g - o) <= 0.002 * o + 5, (g, o)
    tally.close()


def test_energy_ledger_heterogeneous_with_pairs():
    w = _column_workload(32, 0.5, nxy=32, vxy=0.5)
    w.phantom = inputs.slab_phantom(2, 32, 0.5)
    w.phantom.origin = (0.0, 0.0, 0.0)
    dw = engine.upload(w)
    n = 20000
    t, lg = transport_particles(dw, *_pencil(n, 0, 6.0, 8.0, 8.0), seed=5)
    assert lg[5] > 0 and lg[7] == 0
    emitted = n * 6.0 * FP
    assert abs(int(lg[2]) + int(lg[1]) - emitted) <= 1e-6 * emitted
    assert int(t.sum()) == int(lg[2])


def _event_parity(w, n_hist, first=0, min_match=0.97):
    """Per-history comparison on the same Philox streams."""
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    ost = source.psl_build(w.records, w.binning)
    opl = source.make_plan(ost, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)
    hs = np.arange(first, first + n_hist)
    s = source.source(opl, ost, w.records, w.beams, w.phantom, hs, w.z_psl, w.sad)
    m = s.status == source.ST_TRANSPORT
    _, lgo, ho = oracle.transport(s.ptype[m], s.pos[m], s.dir[m], s.e[m], s.wt[m].astype(float),
                                  hs[m].astype(np.uint64), w.phantom, w.seed, per_history=True)
    batch = capi.psl_source_batch(plan, dw.phantom, first, n_hist)
    tally = capi.psl_tally_create(dw.phantom, 1)
    hd = torch.zeros(n_hist, dtype=torch.int64, device="cuda")
    he = torch.zeros(n_hist, dtype=torch.int64, device="cuda")
    hv = torch.zeros(n_hist, dtype=torch.int32, device="cuda")
    capi.transport_trace(dw.phantom, capi.physics(), batch, tally, 0, hd, he, hv)
    gd, ge, gv = hd.cpu().numpy()[m], he.cpu().numpy()[m], hv.cpu().numpy()[m]
    od, oe, ov = ho["dep"], ho["esc"], ho["events"]
    tot_g = (gd + ge).astype(float)
    match = (np.abs(gd - od) <= 1e-4 * np.maximum(tot_g, 1.0) + 16) & (gv == ov)
    # every history conserves its own energy on the GPU
    e_in = np.rint(s.e[m] * s.wt[m].astype(float) * FP)
    assert np.all(np.abs(tot_g - e_in) <= 1e-5 * e_in + 64)
    return match.mean(), match


def test_brute_force_ten_histories():
    w = inputs.config1()
    rate, match = _event_parity(w, 10)
    assert rate >= 0.9


def test_event_parity_config1_block():
    w = inputs.config1()
    rate, _ = _event_parity(w, 3000, first=40_000)
    assert rate >= 0.97


def test_event_parity_config2_sampled():
    """Full-size 1e8-history plan, a sampled range deep inside it."""
    w = inputs.config2()
    rate, _ = _event_parity(w, 2000, first=63_000_000)
    assert rate >= 0.95


@pytest.mark.parametrize("cfg", [3, 4])
def test_event_parity_full_size_ct_plans_sampled(cfg):
    """Full-size CT plans (30x30 field with jaws and fluence, 4e7 records,
    1e9 histories; IMRT plan of 218 segments, 5e8 histories): per-history
    parity on a range deep inside each plan."""
    w = inputs.config3() if cfg == 3 else inputs.config4()
    rate, _ = _event_parity(w, 3000, first=w.n_histories * 3 // 5)
    assert rate >= 0.95


def test_dose_parity_config1():
    w = inputs.config1()
    dw = engine.upload(w)
    g = engine.run(dw)
    torch.cuda.synchronize()
    nz, ny, nx = w.phantom.shape
    dg, sg = g["dose"].cpu().numpy().reshape(nz, ny, nx), g["sigma"].cpu().numpy().reshape(nz, ny, nx)
    o = oracle.run_plan(w)
    do, so = readout.dose(o["tallies"], w.phantom.rho, w.phantom.voxel, g["norm"])
    m = do > 0.1 * do.max()
    rel = np.abs(dg[m] - do[m]).mean() / do[m].mean()
    assert rel < 0.005
    within = np.abs(dg[m] - do[m]) <= 3 * np.sqrt(sg[m] ** 2 + so[m] ** 2)
    assert within.mean() >= 0.99
    gamma, _ = readout.gamma_pass_rate(do, dg, w.phantom.voxel)
    assert gamma >= 0.99
    # energy ledger on the GPU, FP64 sums of the fixed-point counters
    lg = g["ledger"].cpu().numpy()
    assert abs(lg[2] + lg[1] - lg[0]) <= 1e-6 * lg[0]


def test_determinism_and_batch_split():
    w = inputs.config1(n_histories=30_000)
    dw = engine.upload(w)
    a = engine.run(dw, n_batches=1, readout=False)
    ta, la = engine.raw_tallies(dw, a["tally"], 1)
    b = engine.run(dw, n_batches=3, readout=False, store=a["store"], plan=a["plan"])
    tb, lb = engine.raw_tallies(dw, b["tally"], 3)
    assert np.array_equal(ta[0], tb.sum(0))
    assert np.array_equal(la[:7], lb[:7])
    c = engine.run(dw, n_batches=1, readout=False, store=a["store"], plan=a["plan"])
    tc, _ = engine.raw_tallies(dw, c["tally"], 1)
    assert np.array_equal(ta, tc)
    # the slices do not depend on how the range is cut into source batches
    d = engine.run(dw, n_batches=3, readout=False, store=a["store"], plan=a["plan"], batch_size=7_777)
    td, _ = engine.raw_tallies(dw, d["tally"], 3)
    assert np.array_equal(tb, td)


def test_history_slices_follow_the_oracle_partition():
    """PSL_SLICE_BY_HISTORY: every history's deposits land in the batch the
    oracle draws for its id (per-history sums from a traced transport)."""
    w = inputs.config1()
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    n, first, nb = 20_000, 3_000, 7
    batch = capi.psl_source_batch(plan, dw.phantom, first, n)
    tally = capi.psl_tally_create(dw.phantom, nb)
    hd = torch.zeros(n, dtype=torch.int64, device="cuda")
    capi.transport_trace(dw.phantom, capi.physics(), batch, tally, capi.SLICE_BY_HISTORY, hd, None, None)
    t, _ = engine.raw_tallies(dw, tally, nb)
    sl = oracle.history_slices(np.arange(first, first + n), w.seed, nb)
    dep = hd.cpu().numpy()
    for b in range(nb):
        assert int(t[b].sum()) == int(dep[sl == b].sum())
    assert np.all(t.reshape(nb, -1).sum(1) > 0)


def test_batch_uncertainty_falls_as_one_over_root_n():
    """The isocentre batch uncertainty of the 10x10 plan at 1e8 and 4e8
    histories: sigma/D halves (it would plateau if a batch sampled only a
    subset of the PSLs)."""
    w = inputs.config2()
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    nz, ny, nx = w.phantom.shape
    iso = np.array(w.beams[0].iso) - np.array(w.phantom.origin)
    ic = (iso / np.array(w.phantom.voxel)).astype(int)[::-1]
    sl = tuple(slice(c - 2, c + 3) for c in ic)
    rel = []
    for n in (100_000_000, 400_000_000):
        plan = capi.psl_plan_create(store, dw.beams, w.sad, n, w.seed)
        tally = capi.psl_tally_create(dw.phantom, 10)
        capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, n)
        dose = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
        sig = torch.empty_like(dose)
        lg = torch.empty(3, dtype=torch.float64, device="cuda")
        _, n_total, _ = plan.info()
        capi.dose_readout(tally, dw.phantom, engine.normalisation(plan, n), dose, sig, lg)
        d = dose.view(nz, ny, nx).cpu().numpy()
        s = sig.view(nz, ny, nx).cpu().numpy()
        rel.append(float((s[sl] / d[sl]).mean()))
    assert 1.6 < rel[0] / rel[1] < 2.5, rel


def _tallies_of(dw, tally, nb):
    t, lg = engine.raw_tallies(dw, tally, nb)
    return t, lg


@pytest.mark.parametrize("cfg", [1, 4])
def test_psl_run_and_graph_match_per_batch_path(cfg):
    """All histories in one call (no host synchronisation) and as one
    CUDA-graph launch give the same integer tallies, slice by slice, as
    psl_source_batch + transport_run piece by piece."""
    w = inputs.config1(n_histories=60_000) if cfg == 1 else inputs.config4(n_records=300_000, n_histories=200_000)
    w.n_batches = 4
    dw = engine.upload(w)
    ref = engine.run(dw, readout=False)
    t_ref, l_ref = _tallies_of(dw, ref["tally"], 4)
    phys = capi.physics()
    tally = capi.psl_tally_create(dw.phantom, 4)
    capi.psl_run(ref["plan"], dw.phantom, phys, tally, 0, w.n_histories, use_graph=False)
    t1, l1 = _tallies_of(dw, tally, 4)
    assert np.array_equal(t1, t_ref) and np.array_equal(l1[:11], l_ref[:11])
    for _ in range(2):                                   # capture once, replay
        capi.psl_tally_reset(tally)
        capi.psl_run(ref["plan"], dw.phantom, phys, tally, 0, w.n_histories, use_graph=True)
        t2, l2 = _tallies_of(dw, tally, 4)
        assert np.array_equal(t2, t_ref) and np.array_equal(l2[:11], l_ref[:11])
    emitted, escaped, deposited = l2[0], l2[1], l2[2]
    assert abs(int(deposited) + int(escaped) - int(emitted)) <= 1e-6 * emitted


def test_autotune_picks_a_candidate_and_clears_the_tally():
    w = inputs.config1(n_histories=200_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, 10)
    g, d = capi.psl_autotune(plan, dw.phantom, capi.physics(), tally, 100_000)
    # (a 2e5-history plan: depths above its histories, 2^22 ... 2^26, are not tried)
    assert g in (2, 3, 4, 6) and d == 1 << 21
    t, lg = _tallies_of(dw, tally, 10)
    assert t.sum() == 0 and lg[:11].sum() == 0
    # the tuned settings give the same integers as the defaults
    capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, w.n_histories)
    t1, _ = _tallies_of(dw, tally, 10)
    ref = engine.run(dw, readout=False, store=store, plan=plan)
    t2, _ = _tallies_of(dw, ref["tally"], 10)
    assert np.array_equal(t1, t2)


def test_imrt_plan_event_parity_sampled():
    """Multi-segment IMRT plan (config-4 recipe, small phase space): per-history
    parity with the oracle on a sampled range."""
    w = inputs.config4(n_records=300_000, n_histories=1_000_000)
    rate, _ = _event_parity(w, 1500, first=400_000)
    assert rate >= 0.95


@pytest.mark.parametrize("graph", [False, True])
def test_batch_order_gives_the_reading_order_tally(graph):
    """psl_run batch by batch (PSL_ORDER_BATCH: a window's histories sorted
    by batch, one tally slice hot at a time) and in reading order give the
    same tallies and ledger bit for bit, with and without the CUDA graph."""
    nb = 7
    w = inputs.config4(n_records=300_000, n_histories=400_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    phys = capi.physics()
    out = []
    for order in (capi.ORDER_READING, capi.ORDER_BATCH):
        tally = capi.psl_tally_create(dw.phantom, nb)
        capi.psl_tally_set_order(tally, order)
        for _ in range(2 if graph else 1):              # a graph is captured once, then replayed
            capi.psl_tally_reset(tally)
            capi.psl_run(plan, dw.phantom, phys, tally, 1000, w.n_histories - 1000, use_graph=graph)
        out.append(_tallies_of(dw, tally, nb))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1][:11], out[1][1][:11])
    assert out[0][0].sum() > 0


def test_batch_order_windows_on_the_full_imrt_plan():
    """The full IMRT plan (5e8 histories, 10 batches, a 131 MB tally): the
    automatic order runs it batch by batch over 3 windows of ~1.7e8
    histories; the tally equals the reading-order one bit for bit."""
    w = inputs.config4()
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    phys = capi.physics()
    out = []
    for order in (capi.ORDER_AUTO, capi.ORDER_READING):
        tally = capi.psl_tally_create(dw.phantom, w.n_batches)
        capi.psl_tally_set_order(tally, order)
        capi.psl_run(plan, dw.phantom, phys, tally, 0, w.n_histories)
        out.append(_tallies_of(dw, tally, w.n_batches))
        tally.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1][:11], out[1][1][:11])


def test_plan_replay_graph_equals_run_and_readout():
    """psl_plan_replay (tally reset + psl_run + dose_readout recorded as one
    CUDA graph) gives, on every replay, the dose, sigma and ledger of the
    same calls made one by one."""
    w = inputs.config4(n_records=300_000, n_histories=300_000)
    w.n_batches = 5
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    phys = capi.physics()
    nvox = dw.mat_t.numel()
    norm = engine.normalisation(plan, w.n_histories)
    ref = [torch.empty(nvox, dtype=torch.float64, device="cuda") for _ in range(2)] + \
        [torch.empty(3, dtype=torch.float64, device="cuda")]
    t1 = capi.psl_tally_create(dw.phantom, w.n_batches)
    capi.psl_run(plan, dw.phantom, phys, t1, 0, w.n_histories)
    capi.dose_readout(t1, dw.phantom, norm, *ref)
    t2 = capi.psl_tally_create(dw.phantom, w.n_batches)
    out = [torch.full_like(ref[0], -1.0), torch.full_like(ref[1], -1.0), torch.full_like(ref[2], -1.0)]
    for _ in range(3):                                     # record, then two replays
        for o in out:
            o.fill_(-1.0)
        capi.psl_plan_replay(plan, dw.phantom, phys, t2, 0, w.n_histories, norm, *out)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
    assert float(ref[0].sum()) > 0


def test_bin_size_autotuner_picks_a_candidate():
    w = inputs.config2(n_records=1_000_000, n_histories=2_000_000)
    dw = engine.upload(w)
    cells = [0.5, 1.0, 2.0]
    best, secs = capi.psl_autotune_bins(dw.params, dw.records, dw.beams, w.sad, dw.phantom, capi.physics(),
                                        w.n_histories, w.seed, 10, cells, 400_000)
    assert best in cells and np.all(secs > 0) and secs[cells.index(best)] == secs.min()
    with pytest.raises(capi.PslError):
        capi.psl_autotune_bins(dw.params, dw.records, dw.beams, w.sad, dw.phantom, capi.physics(),
                               w.n_histories, w.seed, 10, [0.0], 1000)


def test_traced_and_production_instances_give_the_same_tally():
    """transport_trace launches the kernels' instances that record per-history
    sums; transport_run the production instances compiled without that
    record.  The same source batch must give the same integer tally and
    ledger through both."""
    w = inputs.config1(n_histories=50_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    n = w.n_histories
    got = []
    for traced in (False, True):
        batch = capi.psl_source_batch(plan, dw.phantom, 0, n)
        tally = capi.psl_tally_create(dw.phantom, 1)
        if traced:
            hd = torch.zeros(n, dtype=torch.int64, device="cuda")
            he = torch.zeros(n, dtype=torch.int64, device="cuda")
            hv = torch.zeros(n, dtype=torch.int32, device="cuda")
            capi.transport_trace(dw.phantom, capi.physics(), batch, tally, 0, hd, he, hv)
        else:
            capi.transport_run(dw.phantom, capi.physics(), batch, tally, 0)
        got.append(_tallies_of(dw, tally, 1))
        tally.close()
        batch.close()
    (t1, l1), (t2, l2) = got
    assert t1.sum() > 0
    assert np.array_equal(t1, t2)
    assert np.array_equal(l1, l2)
    # the per-history record adds up to the tally
    assert int(hd.sum().item()) == int(t2.sum())
