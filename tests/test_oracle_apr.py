"""Pins of the oracle's azimuthal particle redistribution (Sec. 2.3.1).

Redistribution rotates a record about the beam axis by a uniform azimuth,
position and direction together.  What fixes it, independently of the code:
the rotation invariants (radius, the in-plane dot and cross products of
position and direction), the doubled-angle identity behind the angle
sampler, uniformity of the angle, and the latent-variance closed forms of
two statistics of a cylindrically symmetric phase space.
"""
import math

import numpy as np
import pytest

from oracle import _lib, source
from paper_1302_1861_b300 import inputs


def _disc_records(rng, n, radius=5.0):
    r = radius * np.sqrt(rng.random(n))
    t = 2 * np.pi * rng.random(n)
    x, y = (r * np.cos(t)).astype(np.float32), (r * np.sin(t)).astype(np.float32)
    d = np.sqrt(x.astype(np.float64) ** 2 + y.astype(np.float64) ** 2 + 100.0 ** 2)
    u, v = (x / d).astype(np.float32), (y / d).astype(np.float32)
    e = rng.uniform(0.1, 6.0, n).astype(np.float32)
    wt = np.ones(n, np.float32)
    q = np.where(rng.random(n) < 0.05, -1, 0).astype(np.int8)
    return inputs.Records(x, y, u, v, e, wt, q)


def test_one_copy_is_the_phase_space_itself():
    w = inputs.config1(n_records=3000)
    r = source.apr_expand(w.records, 1, 99)
    for a, b in zip(r.arrays(), w.records.arrays()):
        assert np.array_equal(a, b)


def test_copy_zero_unchanged_and_payload_replicated():
    w = inputs.config1(n_records=5000)
    k = 5
    r = source.apr_expand(w.records, k, 1234)
    assert r.n == k * w.records.n
    for name in ("x", "y", "u", "v", "e", "wt", "q"):
        a = getattr(r, name).reshape(-1, k)
        b = getattr(w.records, name)
        assert np.array_equal(np.ascontiguousarray(a[:, 0]).view(np.uint8), b.view(np.uint8)), name   # bit for bit
        if name in ("e", "wt", "q"):
            assert np.array_equal(a, np.repeat(b[:, None], k, 1)), name


def test_rotation_invariants():
    """A common rotation of position and direction keeps |r|, |(u,v)|,
    x u + y v and x v - y u; a rotation of the direction by the opposite
    angle, or of one of them only, changes the last two."""
    w = inputs.config1(n_records=20000)
    k = 6
    r = source.apr_expand(w.records, k, 77)
    x, y, u, v = (np.asarray(getattr(w.records, n), np.float64)[:, None] for n in "xyuv")
    X, Y, U, V = (np.asarray(getattr(r, n), np.float64).reshape(-1, k) for n in "xyuv")
    rad = np.hypot(x, y)
    assert np.max(np.abs(np.hypot(X, Y) - rad) / np.maximum(rad, 1e-6)) < 1e-6
    assert np.max(np.abs(np.hypot(U, V) - np.hypot(u, v))) < 1e-7
    assert np.max(np.abs((X * U + Y * V) - (x * u + y * v))) < 1e-6
    assert np.max(np.abs((X * V - Y * U) - (x * v - y * u))) < 1e-6
    # the copies really move: the azimuth changes for almost every copy
    phi0 = np.arctan2(y, x)
    moved = np.abs(np.angle(np.exp(1j * (np.arctan2(Y[:, 1:], X[:, 1:]) - phi0)))) > 1e-3
    assert moved.mean() > 0.99


def test_angle_is_doubled_angle_of_first_accepted_disc_point():
    """cos, sin against cos(2 theta), sin(2 theta) of the first candidate
    point inside the unit disc, found here with a scalar float64 loop."""
    n, k, seed = 40, 4, 0x1302186100
    cs, sn = source.apr_angles(n, k, seed)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for i in range(n):
        for c in range(1, k):
            found = None
            for blk in range(source.APR_MAX_BLOCKS):
                wds = _lib.philox(np.array([[blk, source.TAG_APR, i, c]], np.uint32), key)[0]
                for h in range(2):
                    a = 2.0 * (((int(wds[2 * h]) >> 9) + 0.5) * 2.0 ** -23) - 1.0
                    b = 2.0 * (((int(wds[2 * h + 1]) >> 9) + 0.5) * 2.0 ** -23) - 1.0
                    if a * a + b * b <= 1.0:
                        found = (a, b)
                        break
                if found:
                    break
            th = math.atan2(found[1], found[0])
            assert abs(float(cs[i, c]) - math.cos(2 * th)) < 1e-6
            assert abs(float(sn[i, c]) - math.sin(2 * th)) < 1e-6
    assert np.all(cs[:, 0] == 1) and np.all(sn[:, 0] == 0)


def test_angles_uniform_and_unit():
    n, k = 4000, 6
    cs, sn = source.apr_angles(n, k, 2024)
    c, s = cs[:, 1:].astype(np.float64), sn[:, 1:].astype(np.float64)
    assert np.max(np.abs(c * c + s * s - 1)) < 1e-6
    ang = np.arctan2(s, c).ravel()
    h, _ = np.histogram(ang, 36, (-np.pi, np.pi))
    expct = len(ang) / 36
    chi2 = float(((h - expct) ** 2 / expct).sum())
    assert chi2 < 80.0, chi2                     # 35 dof: p ~ 2e-5 at 80
    m = len(ang)
    assert abs(c.mean()) < 4 / math.sqrt(2 * m) and abs(s.mean()) < 4 / math.sqrt(2 * m)
    # different seeds give different angles; the same seed the same ones
    cs2, sn2 = source.apr_angles(n, k, 2025)
    assert np.mean(cs2[:, 1:] == cs[:, 1:]) < 0.01
    cs3, _ = source.apr_angles(n, k, 2024)
    assert np.array_equal(cs3, cs)


def test_latent_variance_closed_forms():
    """Latent phase-space variance (Sec. 2.3.1) on a cylindrically symmetric
    phase space of N records, M independent realisations, K copies.

    Half-plane statistic F = (1/K) sum over copies of [x > 0]: every copy's
    indicator is an independent Bernoulli(1/2), so Var F = N / (4K), against
    N / 4 for plain recycling (each record K times).  Annulus statistic:
    rotation keeps the radius, so redistribution leaves it unchanged."""
    rng = np.random.default_rng(7)
    n, m, k = 256, 300, 8
    f_apr, f_plain, g_apr, g_plain = [], [], [], []
    for j in range(m):
        rec = _disc_records(rng, n)
        r = source.apr_expand(rec, k, 5000 + j)
        f_apr.append(np.count_nonzero(r.x > 0) / k)
        f_plain.append(np.count_nonzero(rec.x > 0))
        rad2 = r.x.astype(np.float64) ** 2 + r.y.astype(np.float64) ** 2
        g_apr.append(np.count_nonzero((rad2 > 4.0) & (rad2 < 9.0)) / k)
        rad0 = rec.x.astype(np.float64) ** 2 + rec.y.astype(np.float64) ** 2
        g_plain.append(np.count_nonzero((rad0 > 4.0) & (rad0 < 9.0)))
    va, vp = np.var(f_apr, ddof=1), np.var(f_plain, ddof=1)
    tol = 4 * math.sqrt(2.0 / (m - 1))
    assert abs(va / (n / (4 * k)) - 1) < tol, va
    assert abs(vp / (n / 4) - 1) < tol, vp
    assert abs(np.mean(f_apr) - n / 2) < 4 * math.sqrt(n / (4 * k) / m)
    assert np.array_equal(np.array(g_apr), np.array(g_plain, dtype=np.float64))


@pytest.mark.parametrize("k", [2, 3])
def test_psl_build_of_redistributed_phase_space(k):
    """The store of a redistributed phase space against a brute-force stable
    sort of the expanded records' PSL ids."""
    w = inputs.config1(n_records=3000)
    r = source.apr_expand(w.records, k, 31)
    st = source.psl_build(r, w.binning)
    keys = source.psl_keys(r.x, r.y, r.e, r.q, w.binning.x_edges, w.binning.y_edges, w.binning.e_edges)
    idx = sorted(range(r.n), key=lambda i: (keys[i], i))
    idx = [i for i in idx if keys[i] < st.n_bins]
    assert np.array_equal(st.perm, np.array(idx, np.int64))
