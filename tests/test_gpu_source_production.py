"""The production source stage (the source kernel that feeds transport inside
psl_run) against the oracle, bit for bit (Sec. 2.2, 2.3.3, 2.4).

psl_tally_trace_source makes the source kernel of later psl_run calls write
what it decided per history: entry, read number, sorted record, status,
particle type and state.  On the full-size 10x10, 30x30 CT and IMRT plans,
ranges of histories that straddle energy-division (group) boundaries and
the points inside a group where an entry runs out of histories (segment
boundaries: the reading order's round width changes there) are run through
psl_run, in reading order and batch by batch (PSL_ORDER_BATCH: the kernel
reads its histories through the window's sorted offset list), and compared
with oracle.source.source.  Bar: every integer and the float32 weight and
energy bit-exact; the rotated / projected state within 2e-5 cm of the
oracle's float64 value (float32 rounding of ~100 cm coordinates).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402

HALF = 96


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def boundaries(opl, rng, n_group=6, n_seg=10):
    """History ids at group starts and at segment boundaries inside groups:
    in group g (entries with counts c_e, visited by decreasing count), round
    r reads one history from every entry with c_e > r, so the width of the
    rounds changes after sum_e min(c_e, v) histories for every distinct
    count v."""
    gs = opl.group_start
    groups = [g for g in range(len(gs) - 1) if gs[g + 1] > gs[g]]
    out = [int(gs[g]) for g in rng.choice(groups[1:], min(n_group, len(groups) - 1), replace=False)]
    segs = []
    for g in groups:
        c = np.sort(opl.count[opl.group_order[g]])[::-1]
        vals = np.unique(c)[:-1]                 # the largest count ends the group
        for v in vals:
            segs.append(int(gs[g] + np.minimum(c, v).sum()))
    segs = np.array(sorted(set(segs) - set(int(x) for x in gs)))
    if len(segs):
        out += [int(x) for x in rng.choice(segs, min(n_seg, len(segs)), replace=False)]
    return sorted(set(out))


def traced_run(dw, plan, tally, h0, n, order):
    d = dict(entry=torch.full((n,), -1, dtype=torch.int64, device="cuda"),
             use=torch.full((n,), -1, dtype=torch.int64, device="cuda"),
             rec=torch.full((n,), -1, dtype=torch.int64, device="cuda"),
             status=torch.full((n,), -1, dtype=torch.int8, device="cuda"),
             state=torch.zeros(n * 8, dtype=torch.float32, device="cuda"),
             ptype=torch.full((n,), -1, dtype=torch.int32, device="cuda"))
    capi.psl_tally_set_order(tally, order)
    capi.psl_tally_trace_source(tally, h0, n, **d)
    capi.psl_tally_reset(tally)
    capi.psl_run(plan, dw.phantom, capi.physics(), tally, h0, n)
    capi.psl_tally_trace_source(tally, 0, 0)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in d.items()}
    out["state"] = out["state"].reshape(n, 8)
    return out


def check(g, o):
    assert np.array_equal(g["entry"], o.entry) and np.array_equal(g["use"], o.use)
    assert np.array_equal(g["rec"], o.rec)
    assert np.array_equal(g["status"], o.status)
    ok = o.status == source.ST_TRANSPORT
    assert np.array_equal(g["ptype"][ok], o.ptype[ok])
    assert np.array_equal(g["state"][ok, 7], o.wt[ok])                       # weight bit-exact
    assert np.array_equal(g["state"][ok, 6], o.e[ok].astype(np.float32))
    assert np.abs(g["state"][ok, 0:3] - o.pos[ok]).max(initial=0) < 2e-5 * 100
    assert np.abs(g["state"][ok, 3:6] - o.dir[ok]).max(initial=0) < 2e-6
    return int(ok.sum())


@pytest.mark.parametrize("cfg", [2, 3, 4])
def test_production_source_stage_bit_exact_at_boundaries(cfg):
    w = {2: inputs.config2, 3: inputs.config3, 4: inputs.config4}[cfg]()
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    ost = source.psl_build(w.records, w.binning)
    opl = source.make_plan(ost, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)
    tally = capi.psl_tally_create(dw.phantom, w.n_batches)
    rng = np.random.default_rng(100 + cfg)
    starts = [max(0, b - HALF) for b in boundaries(opl, rng)] + [0, w.n_histories - 2 * HALF]
    n_ok = 0
    for h0 in starts:
        hs = np.arange(h0, h0 + 2 * HALF)
        o = source.source(opl, ost, w.records, w.beams, w.phantom, hs, w.z_psl, w.sad)
        for order in (capi.ORDER_READING, capi.ORDER_BATCH):
            n_ok += check(traced_run(dw, plan, tally, h0, 2 * HALF, order), o)
    assert n_ok > 0
    tally.close(); plan.close(); store.close()
