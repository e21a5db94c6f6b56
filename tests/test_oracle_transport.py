"""Pins of the oracle's transport, tally and readout (CPU only).

Closed forms and invariants that fix the transport loop independently of its
code: narrow-beam attenuation exp(-mu x) through one and two materials
(Woodcock tracking), interaction-channel frequencies mu_c/mu, the CSDA range
of an electron with hard events and scattering off, confinement of energy to
the track, the energy ledger, and determinism of the integer tally under any
thread count or history split (Sec. 2.3.3: dose counters, batches).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import _lib, readout, source
from paper_1302_1861_b300 import inputs

L = _lib.lib()


def _pencil(n, ptype, E, phantom, x=0.5, y=0.5):
    pos = np.tile([x, y, 0.0], (n, 1))
    d = np.tile([0.0, 0.0, 1.0], (n, 1))
    return (np.full(n, ptype, np.int32), pos, d, np.full(n, E), np.ones(n), np.arange(n, dtype=np.uint64))


def _column(nz, vz, rho=None, mat=None):
    m = np.zeros((nz, 1, 1), np.uint8) if mat is None else mat
    r = np.ones((nz, 1, 1), np.float32) if rho is None else rho
    return inputs.Phantom(m, r, (1.0, 1.0, vz), (0.0, 0.0, 0.0))


@pytest.mark.parametrize("E", [0.1, 1.0, 6.0])
def test_narrow_beam_attenuation_water(E):
    ph = _column(40, 1.0)
    n = 200_000
    t, lg = oracle.transport(*_pencil(n, 0, E, ph), ph, seed=11, flags=oracle.F_FIRST_INTERACTION)
    mu = L.ora_mu_rho(E, 0, 3)
    # fraction with first interaction beyond depth z: exp(-mu z)
    first = t[:, 0, 0] / (E * 2.0 ** 32)
    beyond = n - np.cumsum(first)
    z = np.arange(1, 41, dtype=float)
    p = np.exp(-mu * z)
    sd = np.sqrt(n * p * (1 - p)) + 1
    assert (np.abs(beyond - n * p) < 5 * sd).all()
    assert abs(lg[oracle.L_ESCAPED] / (E * 2.0 ** 32) - n * math.exp(-mu * 40)) < 5 * sd[-1]


def test_narrow_beam_attenuation_two_media():
    """Woodcock tracking through water then a bone slab (rho 1.85): the
    uncollided fraction is exp(-sum mu_i x_i)."""
    E = 0.08
    rho = np.ones((30, 1, 1), np.float32)
    mat = np.zeros((30, 1, 1), np.uint8)
    rho[10:16] = 1.85
    mat[10:16] = 1
    ph = _column(30, 0.5, rho, mat)
    n = 200_000
    t, lg = oracle.transport(*_pencil(n, 0, E, ph), ph, seed=12, flags=oracle.F_FIRST_INTERACTION)
    mu_w, mu_b = L.ora_mu_rho(E, 0, 3), 1.85 * L.ora_mu_rho(E, 1, 3)
    depth_mu = np.cumsum(np.where((np.arange(30) >= 10) & (np.arange(30) < 16), mu_b, mu_w) * 0.5)
    p = np.exp(-depth_mu)
    beyond = n - np.cumsum(t[:, 0, 0] / (E * 2.0 ** 32))
    sd = np.sqrt(n * p * (1 - p)) + 1
    assert (np.abs(beyond - n * p) < 5 * sd).all()


@pytest.mark.parametrize("E,mat", [(0.04, 0), (0.04, 1), (6.0, 0), (3.0, 1)])
def test_channel_fractions(E, mat):
    ph = _column(20, 1.0, mat=np.full((20, 1, 1), mat, np.uint8))
    n = 200_000
    _, lg = oracle.transport(*_pencil(n, 0, E, ph), ph, seed=13, flags=oracle.F_FIRST_INTERACTION)
    k = lg[[oracle.L_COMPTON, oracle.L_PHOTO, oracle.L_PAIR]].astype(float)
    tot = k.sum()
    mus = np.array([L.ora_mu_rho(E, mat, c) for c in range(3)])
    p = mus / mus.sum()
    sd = np.sqrt(tot * p * (1 - p)) + 1
    assert (np.abs(k - tot * p) < 5 * sd).all()


@pytest.mark.parametrize("T0,rho", [(2.0, 1.0), (0.9, 0.26), (5.0, 1.85)])
def test_csda_range_of_straight_electron(T0, rho):
    """Hard events and scattering off: the path to the cut-off equals
    integral of dT / (rho S_restricted(T)) from the cut-off to T0."""
    nz = 200
    ph = _column(nz, 0.05, rho=np.full((nz, 1, 1), rho, np.float32))
    n = 4
    t, lg, h = oracle.transport(*_pencil(n, 1, T0, ph), ph, seed=3,
                                flags=oracle.F_NO_MSC | oracle.F_NO_HARD | oracle.F_LOCAL_SECONDARIES,
                                per_history=True)
    f = lambda T: 1.0 / (rho * L.ora_restricted_stopping(T, oracle.WCC, oracle.WCB))
    pts = [p for p in (0.2, 0.4) if oracle.ECUT < p < T0]
    csda, _ = integrate.quad(f, oracle.ECUT, T0, epsrel=1e-12, points=pts or None, limit=200)
    assert np.allclose(h["path"], csda, rtol=1e-6)
    # all energy stays on the track, in the voxels the path crossed
    last = int(math.floor(csda / 0.05))
    assert t[last + 1:].sum() == 0 and (t[:last] > 0).all()
    assert abs((lg[oracle.L_DEPOSITED] - n * T0 * 2.0 ** 32) / (n * T0 * 2.0 ** 32)) < 1e-9


@pytest.mark.parametrize("T0,rho", [(2.0, 1.0), (5.0, 1.85)])
def test_csda_range_of_straight_positron(T0, rho):
    """A positron with hard events and scattering off travels the CSDA range
    of its own (Bhabha) restricted stopping power, then annihilates at rest:
    with secondaries kept local its 2 m c^2 is deposited where it stops."""
    nz = 200
    ph = _column(nz, 0.05, rho=np.full((nz, 1, 1), rho, np.float32))
    n = 4
    t, lg, h = oracle.transport(*_pencil(n, 2, T0, ph), ph, seed=3,
                                flags=oracle.F_NO_MSC | oracle.F_NO_HARD | oracle.F_LOCAL_SECONDARIES,
                                per_history=True)
    f = lambda T: 1.0 / (rho * L.ora_restricted_stopping_pos(T, oracle.WCC, oracle.WCB))
    csda, _ = integrate.quad(f, oracle.ECUT, T0, epsrel=1e-12, points=[0.2], limit=200)
    assert np.allclose(h["path"], csda, rtol=1e-6)
    # the electron's range differs: the species' own tables are used
    fe = lambda T: 1.0 / (rho * L.ora_restricted_stopping(T, oracle.WCC, oracle.WCB))
    assert abs(integrate.quad(fe, oracle.ECUT, T0, points=[0.2, 0.4], limit=200)[0] / csda - 1) > 1e-3
    e_all = n * (T0 + 2 * oracle.ME) * 2.0 ** 32
    assert abs((lg[oracle.L_DEPOSITED] - e_all) / e_all) < 1e-9


@pytest.mark.parametrize("ptype", [1, 2])
def test_hard_collision_rate_on_a_thin_slab(ptype):
    """Electrons collide hard at the Moller rate, positrons at the Bhabha
    rate: 3 MeV particles crossing 0.5 mm of water (scatter-free, hard
    bremsstrahlung off by W_cb above the energy) make, to first order, the
    integral of sigma(T) / S(T) dT over the energy they lose on the way."""
    T0, n, dz = 3.0, 400_000, 0.05
    ph = _column(1, dz)
    wcb = 10.0
    _, lg = oracle.transport(*_pencil(n, ptype, T0, ph), ph, seed=8,
                             flags=oracle.F_NO_MSC | oracle.F_LOCAL_SECONDARIES, wcb=wcb)
    pos = ptype == 2
    S = (lambda T: L.ora_restricted_stopping_pos(T, oracle.WCC, wcb)) if pos else \
        (lambda T: L.ora_restricted_stopping(T, oracle.WCC, wcb))
    R = L.ora_range_pos if pos else L.ora_range
    Rinv = L.ora_range_inv_pos if pos else L.ora_range_inv
    t_exit = Rinv(R(T0, oracle.WCC, wcb) - dz, oracle.WCC, wcb)
    sig = L.ora_bhabha_sigma if pos else L.ora_moller_sigma
    other = L.ora_moller_sigma if pos else L.ora_bhabha_sigma
    expect = n * integrate.quad(lambda T: sig(T, oracle.WCC) / S(T), t_exit, T0)[0]
    wrong = n * integrate.quad(lambda T: other(T, oracle.WCC) / S(T), t_exit, T0)[0]
    got = lg[oracle.L_HARD_COLL]
    assert lg[oracle.L_HARD_BREM] == 0
    # first order: a second hard event on the same track is rare (~1 %)
    assert abs(got - expect) < 5 * math.sqrt(expect) + 0.02 * expect
    assert abs(got - wrong) > 10 * math.sqrt(expect)


def test_energy_deposited_only_along_track():
    ph = inputs.water_phantom(21, 0.5)
    ph.origin = (0.0, 0.0, 0.0)
    n = 50
    pos = np.tile([5.25, 5.25, 0.0], (n, 1))
    args = (np.ones(n, np.int32), pos, np.tile([0.0, 0.0, 1.0], (n, 1)), np.full(n, 3.0), np.ones(n),
            np.arange(n, dtype=np.uint64))
    t, _ = oracle.transport(*args, ph, seed=4, flags=oracle.F_NO_MSC | oracle.F_NO_HARD)
    mask = np.zeros_like(t, bool)
    mask[:, 10, 10] = True
    assert t[~mask].sum() == 0 and t[mask].sum() > 0


def test_energy_ledger_config1():
    """Deposited + escaped = emitted (fixed point, relative 1e-6)."""
    w = inputs.config1(n_records=20000, n_histories=20000)
    r = oracle.run_plan(w)
    lg = r["ledger"]
    assert lg[oracle.L_ERRORS] == 0
    assert abs(lg[oracle.L_DEPOSITED] + lg[oracle.L_ESCAPED] - lg[oracle.L_EMITTED]) <= 1e-6 * lg[oracle.L_EMITTED]
    assert int(r["tallies"].sum()) == int(lg[oracle.L_DEPOSITED])


def test_energy_ledger_heterogeneous_with_pairs():
    # 6 MeV photons through bone and lung: pair production and annihilation
    ph = inputs.slab_phantom(2, 32, 0.5)
    ph.origin = (0.0, 0.0, 0.0)
    n = 5000
    _, lg = oracle.transport(*_pencil(n, 0, 6.0, ph, 8.0, 8.0), ph, seed=5)
    assert lg[oracle.L_PAIR] > 0 and lg[oracle.L_ERRORS] == 0
    assert abs(lg[oracle.L_DEPOSITED] + lg[oracle.L_ESCAPED] - n * 6.0 * 2 ** 32) <= 1e-6 * n * 6.0 * 2 ** 32


def test_tally_independent_of_threads_and_split():
    w = inputs.config1(n_records=10000, n_histories=6000)
    st = source.psl_build(w.records, w.binning)
    pl = source.make_plan(st, w.beams, w.n_histories, w.seed, w.z_psl, w.sad)
    h = np.arange(6000)
    s = source.source(pl, st, w.records, w.beams, w.phantom, h, w.z_psl, w.sad)
    m = s.status == source.ST_TRANSPORT
    args = (s.ptype[m], s.pos[m], s.dir[m], s.e[m], s.wt[m].astype(float), h[m].astype(np.uint64))
    t1, l1 = oracle.transport(*args, w.phantom, w.seed, nthreads=1)
    t8, l8 = oracle.transport(*args, w.phantom, w.seed, nthreads=8)
    assert np.array_equal(t1, t8) and np.array_equal(l1, l8)
    # two shards (history ranges) sum to the same integers: resume/shard invariance
    k = int(m.sum()) // 3
    a = tuple(x[:k] for x in args)
    b = tuple(x[k:] for x in args)
    ta, la = oracle.transport(*a, w.phantom, w.seed)
    tb, lb = oracle.transport(*b, w.phantom, w.seed)
    assert np.array_equal(ta + tb, t1) and np.array_equal(la + lb, l1)


# ------------------------------------------------------------- readout -----
def test_dose_closed_form_and_sigma():
    rho = np.full((2, 2, 2), 0.5, np.float32)
    t = np.zeros((4, 2, 2, 2), np.int64)
    # 1 MeV per batch in voxel (1,0,1) with batch values 1, 2, 3, 2 MeV
    for b, mev in enumerate((1, 2, 3, 2)):
        t[b, 1, 0, 1] = mev * 2 ** 32
    d, s = readout.dose(t, rho, (0.2, 0.2, 0.2), norm=0.5)
    m = 0.5 * 0.008 * 1e-3
    assert d[1, 0, 1] == pytest.approx(8 * 1.602176634e-13 / m * 0.5, rel=1e-14)
    # batch estimates x_b = 4 t_b c: std of the mean = std(x)/sqrt(4)
    x = np.array([1, 2, 3, 2]) * 4 * 1.602176634e-13 / m * 0.5
    assert s[1, 0, 1] == pytest.approx(x.std(ddof=1) / 2, rel=1e-12)
    assert d.sum() == d[1, 0, 1]


def test_gamma_index():
    z = np.arange(40)[:, None, None]
    ref = np.exp(-((z - 20.0) / 6.0) ** 2) * np.ones((40, 8, 8))
    assert readout.gamma_pass_rate(ref, ref, (0.25, 0.25, 0.25))[0] == 1.0
    # a 1 mm shift passes 2%/2mm and fails 2%/0.5mm on the slopes
    sh = np.exp(-((z - 20.4) / 6.0) ** 2) * np.ones((40, 8, 8))
    assert readout.gamma_pass_rate(ref, sh, (0.25, 0.25, 0.25))[0] == 1.0
    assert readout.gamma_pass_rate(ref, sh, (0.25, 0.25, 0.25), dta_cm=0.05)[0] < 0.9
    # on a flat dose a 5 % scale fails 2 % everywhere; a 1.5 % scale passes
    flat = np.ones((10, 10, 10))
    assert readout.gamma_pass_rate(flat, 1.05 * flat, (0.25, 0.25, 0.25))[0] == 0.0
    assert readout.gamma_pass_rate(flat, 1.015 * flat, (0.25, 0.25, 0.25))[0] == 1.0
