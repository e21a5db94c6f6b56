"""Dose parity on the full-size plans (Sec. 2.3.3 dose counters and batches,
Sec. 2.5 readout), in the launch the benchmark times.

The 10x10 slab plan (1e7 records, 1e8 histories), the 30x30 CT plan (4e7
records, jaws and a fluence map, 1e9 histories) and the IMRT plan (218
segments over the same phase space, 5e8 histories) are built whole on both
sides.  The oracle cannot transport a whole plan, so the plan is cut into
equal strata (the reading order visits the energy divisions one after the
other, so the strata span them all) and one history range is drawn inside
each.  The GPU runs exactly those ranges with psl_run into one 10-batch
tally; the oracle runs the same histories on the same Philox streams.

Bars: mean relative difference < 0.5 % over voxels above 10 % of the
maximum; >= 99 % of them within 3 combined batch standard deviations;
gamma 2 %/2 mm >= 99 % (the oracle's gamma); energy ledger deposited +
escaped = emitted within 1e-6.  The maximum and the voxels compared are
those of the body (density >= 0.1 g/cm^3): the air around the CT body
(0.001 g/cm^3) turns one deposit into a dose 1000 times that of tissue, so
a handful of air voxels would otherwise set the maximum (the slab phantom
has no such voxels).  The histories per voxel are chosen so that branches
flipped by FP32-vs-FP64 rounding (a few % of histories) average out below
the bar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import readout, source  # noqa: E402
from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ranges(n_total, n, k, seed):
    """k disjoint ranges of n histories, one at a random place in each of k
    equal strata of the plan."""
    rng = np.random.default_rng(seed)
    width = n_total // k
    return [int(s * width + rng.integers(0, width - n)) for s in range(k)]


def _dose_parity(w, n, k, seed):
    nb = 10
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    tally = capi.psl_tally_create(dw.phantom, nb)
    firsts = _ranges(w.n_histories, n, k, seed)
    phys = capi.physics()
    for f in firsts:
        capi.psl_run(plan, dw.phantom, phys, tally, f, n)
    nz, ny, nx = w.phantom.shape
    dose = torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
    sig = torch.empty_like(dose)
    lg = torch.empty(3, dtype=torch.float64, device="cuda")
    capi.dose_readout(tally, dw.phantom, 1.0, dose, sig, lg)
    torch.cuda.synchronize()
    dg = dose.view(nz, ny, nx).cpu().numpy()
    sg = sig.view(nz, ny, nx).cpu().numpy()
    lg = lg.cpu().numpy()
    del dw, store, plan, tally
    torch.cuda.empty_cache()

    ost = source.psl_build(w.records, w.binning)
    opl = source.make_plan(ost, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)
    tall = np.zeros((nb, nz, ny, nx), np.int64)
    for f in firsts:
        tall += oracle.run_plan(w, n_histories=n, first=f, n_batches=nb, store=ost, plan=opl)["tallies"]
    do, so = readout.dose(tall, w.phantom.rho, w.phantom.voxel, 1.0)

    body = w.phantom.rho >= 0.1
    m = body & (do > 0.1 * do[body].max())
    rel = np.abs(dg[m] - do[m]).mean() / do[m].mean()
    within = (np.abs(dg[m] - do[m]) <= 3 * np.sqrt(sg[m] ** 2 + so[m] ** 2)).mean()
    gamma, nv = readout.gamma_pass_rate(np.where(body, do, 0.0), np.where(body, dg, 0.0), w.phantom.voxel)
    print(f"{w.name}: {k} x {n} histories, {int(m.sum())} voxels > 10 % max: mean rel diff {rel:.2e}, "
          f"within 3 sigma {within:.4f}, gamma 2%/2mm {gamma:.4f} ({nv} voxels)")
    assert rel < 0.005
    assert within >= 0.99
    assert gamma >= 0.99
    assert abs(lg[2] + lg[1] - lg[0]) <= 1e-6 * lg[0]


def test_dose_parity_10x10_slab_full_plan():
    _dose_parity(inputs.config2(), 100_000, 6, 21)


def test_dose_parity_30x30_ct_full_plan():
    _dose_parity(inputs.config3(), 3_500_000, 6, 31)


def test_dose_parity_imrt_full_plan():
    _dose_parity(inputs.config4(), 400_000, 6, 41)
