"""Degenerate cases of the path on the GPU, each against the oracle or a
closed form (Sec. 2.3.3 selection and counts, Sec. 2.5 readout):

* a field whose region of interest meets no PSL: the plan is refused on
  both sides (PSL_EINVAL / ValueError);
* a phantom of one voxel: the source stage and transport run, energy is
  conserved, and the voxel's tally matches the oracle's;
* a phantom every history misses: nothing is deposited, everything emitted
  is escaped, on both sides;
* one history at each end of a plan, and an empty caller batch;
* a transport workspace kept from a destroyed tally (for a smaller phantom)
  gives the same tally as a fresh one.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402

@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(w, nb=2, first=0, n=None):
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, nb)
    n = w.n_histories if n is None else n
    capi.psl_run(plan, dw.phantom, capi.physics(), tally, first, n)
    t, lg = engine.raw_tallies(dw, tally, nb)
    return t, lg


def test_field_outside_the_phase_space_selects_no_psl():
    w = inputs.config1(n_records=5000, n_histories=1000)
    w.beams = [dataclasses.replace(w.beams[0], x1=30.0, x2=34.0, y1=30.0, y2=34.0)]
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    with pytest.raises(capi.PslError):
        capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    ost = source.psl_build(w.records, w.binning)
    with pytest.raises(ValueError):
        source.make_plan(ost, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)


def test_one_voxel_phantom():
    w = inputs.config1(n_records=20_000, n_histories=20_000)
    # one 20 cm voxel of water around the isocentre, its surface at SSD 90
    w.phantom = inputs.Phantom(np.zeros((1, 1, 1), np.uint8), np.ones((1, 1, 1), np.float32), (20.0, 20.0, 20.0),
                               (-10.0, -10.0, 90.0))
    t, lg = _run(w, nb=2)
    assert lg[2] > 0
    assert abs(int(lg[2]) + int(lg[1]) - int(lg[0])) <= 1e-6 * lg[0]
    o = oracle.run_plan(w, n_batches=2)
    tg, to = t.sum(0).astype(float), o["tallies"].sum(0).astype(float)
    assert tg.shape == to.shape == (1, 1, 1)
    assert abs(tg[0, 0, 0] - to[0, 0, 0]) <= 2e-3 * to[0, 0, 0]


def test_phantom_every_history_misses():
    w = inputs.config1(n_records=20_000, n_histories=20_000)
    ph = w.phantom
    w.phantom = inputs.Phantom(ph.mat, ph.rho, ph.voxel, (ph.origin[0] + 200.0, ph.origin[1], ph.origin[2]))
    t, lg = _run(w, nb=2)
    assert int(t.sum()) == 0 and int(lg[2]) == 0
    assert int(lg[1]) == int(lg[0]) > 0
    o = oracle.run_plan(w, n_batches=2)
    assert int(o["tallies"].sum()) == 0
    assert abs(int(o["ledger"][0]) - int(lg[0])) <= 1e-6 * int(lg[0])        # emitted (FP32 vs FP64 weights)


@pytest.mark.parametrize("where", ["first", "last"])
def test_single_history_runs(where):
    w = inputs.config1(n_records=20_000, n_histories=5_000)
    first = 0 if where == "first" else w.n_histories - 1
    t, lg = _run(w, nb=2, first=first, n=1)
    assert abs(int(lg[2]) + int(lg[1]) - int(lg[0])) <= 1e-6 * max(int(lg[0]), 1) + 64
    o = oracle.run_plan(w, n_histories=1, first=first, n_batches=2)
    assert abs(int(o["ledger"][0]) - int(lg[0])) <= 1e-6 * max(int(lg[0]), 1) + 16
    tg, to = int(t.sum()), int(o["tallies"].sum())
    assert abs(tg - to) <= 1e-4 * max(to, 1) + 64


def test_empty_caller_batch():
    w = inputs.config1(n_records=100, n_histories=100)
    dw = engine.upload(w)
    state = torch.zeros(0, 8, dtype=torch.float32, device="cuda")
    ptype = torch.zeros(0, dtype=torch.int32, device="cuda")
    pid = torch.zeros(0, dtype=torch.int64, device="cuda")
    batch = capi.psl_batch_from_particles(state, ptype, pid, 7)      # n = 0 is a valid, empty batch
    assert batch.info()[0] == 0
    tally = capi.psl_tally_create(dw.phantom, 1)
    capi.transport_run(dw.phantom, capi.physics(), batch, tally, 0)
    t, lg = engine.raw_tallies(dw, tally, 1)
    assert int(t.sum()) == 0 and int(lg[0]) == 0 and int(lg[2]) == 0


def test_kept_workspace_gives_the_same_tally():
    """A destroyed tally's transport workspace is kept and taken by the next
    tally: here a 32^3 phantom's (so the 64^3 run after it must grow the
    packed-density buffer).  The result equals a run on a fresh workspace,
    bit for bit."""
    capi.memory_trim()                                   # nothing kept from earlier tests
    small = inputs.config1(n_records=20_000, n_histories=300_000)
    big = inputs.config2(n_records=200_000, n_histories=200_000)

    def run(w):
        dw = engine.upload(w)
        store = capi.psl_build(dw.params, dw.records)
        plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
        tally = capi.psl_tally_create(dw.phantom, 2)
        capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, w.n_histories)
        out = engine.raw_tallies(dw, tally, 2)
        tally.close()
        return out

    run(small)                                           # its workspace (room for 300,000 primaries) is kept
    t_kept, l_kept = run(big)                            # ... and taken here
    capi.memory_trim()
    t_fresh, l_fresh = run(big)                          # a new workspace
    assert t_kept.sum() > 0
    assert np.array_equal(t_kept, t_fresh)
    assert np.array_equal(l_kept[:11], l_fresh[:11])
