"""The tally does not depend on the queue depth (primaries per transport
pass, psl_tally_set_queue_depth).

A run cut into many passes hands each pass's secondaries (bremsstrahlung
and annihilation photons, delta rays) to the next pass's photon and electron
launches, and the photon feed serves a pass's primaries and those carried
photons as one index space; every particle keeps its own random stream and
tally slice, so the integers must equal those of a single pass.  Both the
lazy source path (psl_run) and caller particles (transport_run) are cut
into passes of 4096 primaries here.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_1861_b300 import capi, engine, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_psl_run_same_tally_at_any_queue_depth():
    w = inputs.config1(n_histories=100_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    got = []
    for depth in (1 << 24, 1 << 12):
        tally = capi.psl_tally_create(dw.phantom, 4)
        capi.psl_tally_set_queue_depth(tally, depth)
        capi.psl_run(plan, dw.phantom, capi.physics(), tally, 0, w.n_histories)
        got.append(engine.raw_tallies(dw, tally, 4))
        tally.close()
    (t1, l1), (t2, l2) = got
    assert t1.sum() > 0
    assert np.array_equal(t1, t2)
    assert np.array_equal(l1, l2)


def test_caller_particles_same_tally_at_any_queue_depth():
    """Photons and electrons of a caller batch (the feed's first queue and the
    electron queue), transported in one pass and in passes of 4096."""
    w = inputs.config1(n_histories=1000)
    dw = engine.upload(w)
    rng = np.random.default_rng(5)
    n = 20_000
    nx, ny, nz = w.phantom.shape[2], w.phantom.shape[1], w.phantom.shape[0]
    vx, vy, vz = w.phantom.voxel
    pos = np.stack([rng.uniform(0.3, 0.7, n) * nx * vx, rng.uniform(0.3, 0.7, n) * ny * vy,
                    np.full(n, 0.01)], 1).astype(np.float32)
    dirs = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (n, 1))
    ptype = (rng.random(n) < 0.2).astype(np.int32)          # 20 % electrons
    e = np.where(ptype == 0, rng.uniform(0.5, 6.0, n), rng.uniform(0.3, 4.0, n)).astype(np.float32)
    wt = np.ones(n, np.float32)
    state = np.concatenate([pos, dirs, e[:, None], wt[:, None]], 1)
    got = []
    for depth in (1 << 24, 1 << 12):
        st = torch.from_numpy(np.ascontiguousarray(state)).cuda()
        pt = torch.from_numpy(ptype).cuda()
        pd = torch.from_numpy(np.arange(n, dtype=np.int64)).cuda()
        batch = capi.psl_batch_from_particles(st, pt, pd, w.seed)
        tally = capi.psl_tally_create(dw.phantom, 1)
        capi.psl_tally_set_queue_depth(tally, depth)
        capi.transport_run(dw.phantom, capi.physics(), batch, tally, 0)
        got.append(engine.raw_tallies(dw, tally, 1))
        tally.close()
        batch.close()
    (t1, l1), (t2, l2) = got
    assert t1.sum() > 0
    assert np.array_equal(t1, t2)
    assert np.array_equal(l1, l2)
