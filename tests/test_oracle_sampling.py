"""Pins of the oracle's sampling steps that the energy ledger cannot see
(CPU only).

The ledger conserves energy whatever angle or split is drawn, so each step
below is checked against the mathematics that defines it, not against the
oracle's own expression: Highland's angle recomputed from the particle's
momentum and checked against a hand computation; the multiple-scattering
polar angle against its Rayleigh law; the direction rotation by its
invariants (unit length, the polar cosine, the azimuth turning with phi, a
uniform azimuth about the old direction), including the branch for
directions along z; the hard bremsstrahlung photon against the 1/k
spectrum; the pair split against the uniform law; the annihilation photons
for isotropy and exact opposition.  The transport loop calls these very
functions (Sec. 2.3.3 hands particles to class-II condensed-history
transport; the photon cut-offs and electron cut-offs are those of Sec. 2.6).
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import _lib

L = _lib.lib()
P = _lib._p
ME = 0.51099895
X0 = 36.08           # radiation length of water, g/cm^2


def chi2_sf(obs, p):
    n = obs.sum()
    e = n * np.asarray(p)
    return stats.chi2.sf(((obs - e) ** 2 / e).sum(), len(p) - 1)


# --------------------------------------------------------------- Highland --
def highland_by_momentum(T, s, rho):
    """Highland's theta0 = 13.6 MeV / (beta p c) sqrt(x/X0) (1 + 0.038 ln(x/X0)),
    with p c and beta taken from the total energy E = T + m c^2."""
    E = T + ME
    pc = math.sqrt(E * E - ME * ME)
    beta = pc / E
    t = s * rho / X0
    return 13.6 / (beta * pc) * math.sqrt(t) * (1.0 + 0.038 * math.log(t))


@pytest.mark.parametrize("T,s,rho", [(1.0, 0.1, 1.0), (5.0, 0.25, 1.85), (0.3, 0.02, 0.26), (12.0, 1.0, 1.04)])
def test_highland_against_momentum_form(T, s, rho):
    assert L.ora_highland(T, s, rho) == pytest.approx(highland_by_momentum(T, s, rho), rel=1e-12)


def test_highland_hand_value_and_density_scaling():
    # by hand, T = 1 MeV, 1 mm of water: E = 1.511 MeV, pc = 1.4220 MeV,
    # beta = 0.9411, beta pc = 1.3382 MeV; x/X0 = 0.1/36.08 = 2.7716e-3,
    # sqrt = 0.052646, 1 + 0.038 ln = 0.77624: theta0 = 0.4153 rad
    assert L.ora_highland(1.0, 0.1, 1.0) == pytest.approx(0.4153, rel=2e-4)
    # X0 scales with density: a step of s at rho is a step of s rho at 1
    for T in (0.5, 3.0):
        assert L.ora_highland(T, 0.2, 0.25) == pytest.approx(L.ora_highland(T, 0.05, 1.0), rel=1e-12)
    # a step too short for the logarithmic correction gives no deflection
    assert L.ora_highland(1.0, 1e-14, 1.0) == 0.0
    assert L.ora_highland(1.0, 0.0, 1.0) == 0.0


def test_msc_polar_angle_is_rayleigh_and_azimuth_uniform():
    n, th0 = 400_000, 0.07
    th, ph = np.zeros(n), np.zeros(n)
    L.ora_sample_msc(th0, 31, n, P(th), P(ph))
    # Rayleigh CDF 1 - exp(-theta^2 / (2 theta0^2)): 40 bins of equal probability
    q = np.linspace(0, 1, 41)
    edges = th0 * np.sqrt(-2.0 * np.log1p(-q[:-1]))
    edges = np.append(edges, np.inf)
    obs, _ = np.histogram(th, edges)
    assert chi2_sf(obs, np.full(40, 1 / 40)) > 1e-3
    assert np.mean(th ** 2) == pytest.approx(2 * th0 ** 2, rel=0.01)       # E[theta^2] = 2 theta0^2
    obs, _ = np.histogram(ph, np.linspace(0, 2 * math.pi, 37))
    assert chi2_sf(obs, np.full(36, 1 / 36)) > 1e-3


# --------------------------------------------------------------- rotation --
def _frame(d):
    """Two unit vectors completing d to an orthonormal right-handed frame."""
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(d, a)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(d, e1)


def _rotate(d, c, phi):
    n = len(c)
    din = np.ascontiguousarray(np.tile(d, (n, 1)))
    out = np.zeros((n, 3))
    L.ora_rotate(n, P(din), P(np.ascontiguousarray(c, float)), P(np.ascontiguousarray(phi, float)), P(out))
    return out


@pytest.mark.parametrize("d", [
    [0.3, -0.4, math.sqrt(1 - 0.25)],          # general
    [0.0, 0.6, -0.8],
    [1e-3, -2e-3, math.sqrt(1 - 5e-6)],        # |w| > 0.99999: the branch along z
    [0.0, 0.0, -1.0],
])
def test_rotation_invariants(d):
    d = np.array(d, float)
    d /= np.linalg.norm(d)
    rng = np.random.default_rng(5)
    n = 20_000
    c = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    out = _rotate(d, c, phi)
    assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-12)
    assert np.allclose(out @ d, c, atol=1e-9)
    # the azimuth about d turns with phi at unit rate (one sense for all phi):
    # a rotation, so a uniform phi gives a uniform azimuth about d
    e1, e2 = _frame(d)
    az = np.arctan2(out @ e2, out @ e1)
    keep = np.abs(c) < 0.999                   # azimuth defined
    for sgn in (1.0, -1.0):
        r = np.angle(np.exp(1j * (az - sgn * phi)))[keep]
        if np.abs(np.angle(np.exp(1j * (r - r[0])))).max() < 1e-5:
            break
    else:
        pytest.fail("azimuth is not phi plus a constant")
    obs, _ = np.histogram(az[keep], np.linspace(-math.pi, math.pi, 25))
    assert chi2_sf(obs, np.full(24, 1 / 24)) > 1e-3


# ---------------------------------------------------------- bremsstrahlung --
@pytest.mark.parametrize("T", [0.5, 2.0, 6.0])
def test_brem_photon_energy_follows_one_over_k(T):
    wcb, n = 0.2, 300_000
    k = np.zeros(n)
    L.ora_sample_brem(T, wcb, 41, n, P(k))
    assert k.min() >= wcb and k.max() <= T
    # 1/k on [wcb, T]: P(k < x) = ln(x/wcb) / ln(T/wcb); 30 bins of equal probability
    edges = wcb * (T / wcb) ** np.linspace(0, 1, 31)
    obs, _ = np.histogram(k, edges)
    assert chi2_sf(obs, np.full(30, 1 / 30)) > 1e-3
    # and not the flat or the 1/k^2 law: the mean of a 1/k law is (T - wcb) / ln(T / wcb)
    assert k.mean() == pytest.approx((T - wcb) / math.log(T / wcb), rel=0.01)


# --------------------------------------------------------- pair production --
@pytest.mark.parametrize("E", [1.5, 6.0])
def test_pair_split_uniform_and_conserving(E):
    n = 200_000
    t1, t2 = np.zeros(n), np.zeros(n)
    L.ora_sample_pair(E, 43, n, P(t1), P(t2))
    avail = E - 2 * ME
    assert np.allclose(t1 + t2, avail, rtol=0, atol=1e-13)
    assert (t1 >= 0).all() and (t2 >= 0).all()
    assert stats.kstest(t1 / avail, "uniform").pvalue > 1e-3
    assert stats.kstest(t2 / avail, "uniform").pvalue > 1e-3


# ------------------------------------------------------------ annihilation --
def test_annihilation_photons_isotropic_and_back_to_back():
    n = 300_000
    d1, d2 = np.zeros(n * 3), np.zeros(n * 3)
    L.ora_sample_annihilation(47, n, P(d1), P(d2))
    d1, d2 = d1.reshape(n, 3), d2.reshape(n, 3)
    assert np.array_equal(d2, -d1)                                   # exactly opposite
    assert np.allclose(np.linalg.norm(d1, axis=1), 1.0, atol=1e-12)
    # isotropic: each Cartesian component is uniform on [-1, 1] (Archimedes),
    # and the azimuth about z is uniform
    for k in range(3):
        obs, _ = np.histogram(d1[:, k], np.linspace(-1, 1, 21))
        assert chi2_sf(obs, np.full(20, 1 / 20)) > 1e-3
    obs, _ = np.histogram(np.arctan2(d1[:, 1], d1[:, 0]), np.linspace(-math.pi, math.pi, 25))
    assert chi2_sf(obs, np.full(24, 1 / 24)) > 1e-3
    assert np.abs(d1.mean(axis=0)).max() < 5 / math.sqrt(n)
