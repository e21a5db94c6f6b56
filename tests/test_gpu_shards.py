"""History-range shards on one GPU (Sec. 2.3.3: histories are independent,
every random stream is keyed by the history id and the dose counters are
integers), the multi-GPU contract of the path exercised on one device.

K shards of one plan's history range, each on its own CUDA stream with its
own tally, must add up bit for bit to the tally of the whole range run at
once; so must the ledgers.  The shards never wait on one another.
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


@pytest.mark.parametrize("k", [2, 3])
def test_stream_shards_sum_to_the_whole_run(k):
    nb = 10
    w = inputs.config2(n_records=500_000, n_histories=3_000_000)
    dw = engine.upload(w)
    store = capi.psl_build(dw.params, dw.records)
    plan = capi.psl_plan_create(store, dw.beams, w.sad, w.n_histories, w.seed)
    phys = capi.physics()
    whole = capi.psl_tally_create(dw.phantom, nb)
    capi.psl_run(plan, dw.phantom, phys, whole, 0, w.n_histories)
    t_whole, l_whole = engine.raw_tallies(dw, whole, nb)

    streams = [torch.cuda.Stream() for _ in range(k)]
    tallies = [capi.psl_tally_create(dw.phantom, nb) for _ in range(k)]
    covered = 0
    for r in range(k):
        first, n, n_plan = engine.shard_histories(r, k, w.n_histories // k)
        assert n_plan == w.n_histories and first == covered
        covered += n
        with torch.cuda.stream(streams[r]):
            capi.psl_run(plan, dw.phantom, phys, tallies[r], first, n, stream=streams[r])
    torch.cuda.synchronize()
    assert covered == w.n_histories
    parts = [engine.raw_tallies(dw, t, nb) for t in tallies]
    t_sum = sum(p[0] for p in parts)
    l_sum = sum(p[1] for p in parts)
    assert np.array_equal(t_sum, t_whole)
    assert np.array_equal(l_sum[:11], l_whole[:11])
    assert t_whole.sum() > 0
