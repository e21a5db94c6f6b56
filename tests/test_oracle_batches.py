"""Pins of the oracle's batch partition (Sec. 2.3.3: independent batches).

Every history belongs to one batch, drawn for its block of 256 consecutive
ids.  What the batch uncertainty needs, checked here: the batch of a block
is uniform over the N_b batches and independent of its neighbours', all
histories of a block share it, and the batch of a history is independent of
the history's position in any periodic reading pattern (the PSL reading
order visits PSLs round-robin, so a batch made of every N_b-th history
would see a fixed subset of PSLs and its spread would not shrink with more
histories).
"""
import numpy as np

import oracle


def _chi2(counts):
    e = counts.sum() / len(counts)
    return float(((counts - e) ** 2 / e).sum())


def test_batches_uniform_and_deterministic():
    h = np.arange(2_000_000, dtype=np.int64) * 263 + 123       # (263 > 256: one history per block)
    s = oracle.history_slices(h, 1302186102, 10)
    assert s.min() >= 0 and s.max() <= 9
    assert _chi2(np.bincount(s, minlength=10)) < 40          # 9 dof, p ~ 4e-6
    assert np.array_equal(s, oracle.history_slices(h, 1302186102, 10))
    s2 = oracle.history_slices(h, 1302186103, 10)
    assert np.mean(s2 == s) < 0.15                            # another seed, another partition


def test_batches_independent_of_periodic_reading_patterns():
    """For every residue of the history id modulo small periods (the widths
    of round-robin reading rounds), the batch is still uniform: no batch is
    tied to a subset of PSLs."""
    h = np.arange(3_000_000, dtype=np.int64)
    s = oracle.history_slices(h, 99, 10)
    for period in (2, 4, 5, 10, 12, 64, 300, 1000):
        for r in range(min(period, 6)):
            # a block gives ~256/period histories of the class (at least one
            # block per history beyond 256): count in units of blocks
            c = np.bincount(s[r::period], minlength=10) / max(1.0, 256.0 / period)
            assert _chi2(c) < 45, (period, r)
    # a block's histories share its batch; consecutive blocks' batches are
    # independent (their joint distribution is flat)
    blocks = s[: len(s) // 256 * 256].reshape(-1, 256)
    assert (blocks == blocks[:, :1]).all()
    b = blocks[:, 0]
    pair = b[:-1] * 10 + b[1:]
    assert _chi2(np.bincount(pair, minlength=100)) < 200      # 99 dof


def test_batches_large_ids():
    h = (np.arange(100_000, dtype=np.int64) * 256 + (1 << 33))   # one history per block, beyond 2^32
    s = oracle.history_slices(h, 5, 1024)
    assert s.min() >= 0 and s.max() <= 1023
    assert _chi2(np.bincount(s, minlength=1024)) < 1300       # 1023 dof
