"""Pins of the oracle's physics formulas and samplers (CPU only).

The paper prints no transport physics (it defers to Jia et al. 2011); the
synthetic model's formulas are pinned here against closed forms and limits
that do not use the oracle's own expressions: the Thomson limit, numerical
integration of the textbook differential cross sections, the unrestricted
Bethe formula in its ICRU Report 37 form, and the identity linking restricted
stopping power to the hard-collision cross section.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from oracle import _lib

L = _lib.lib()
ME = oracle.ME
RE = 2.8179403262e-13
NA = 6.02214076e23
ZA_WATER = 0.555087


def kn_dsigma_domega(E, c):
    """Klein-Nishina differential cross section per electron, cm^2/sr."""
    k = E / ME
    P = 1.0 / (1.0 + k * (1.0 - c))
    return 0.5 * RE * RE * P * P * (P + 1.0 / P - (1.0 - c * c))


# ------------------------------------------------------------ photons -----
def test_kn_thomson_limit():
    sigma_t = 8.0 * math.pi / 3.0 * RE * RE
    k = 1e-3
    series = sigma_t * (1 - 2 * k + 26.0 / 5.0 * k * k)
    assert abs(L.ora_kn_sigma(k * ME) / series - 1) < 1e-5


@pytest.mark.parametrize("E", [0.01, 0.1, 0.5, 1.0, 2.0, 6.0, 20.0])
def test_kn_total_is_integral_of_differential(E):
    num, _ = integrate.quad(lambda c: 2 * math.pi * kn_dsigma_domega(E, c), -1, 1, epsabs=0, epsrel=1e-12)
    assert abs(L.ora_kn_sigma(E) / num - 1) < 1e-9


def test_kn_reference_value_1mev():
    # 1 MeV: about 0.2112 barn per electron (textbook Klein-Nishina value)
    assert abs(L.ora_kn_sigma(1.0) / 2.112e-25 - 1) < 2e-3


@pytest.mark.parametrize("E", [0.1, 1.0, 6.0])
def test_kahn_sampler_chi2(E):
    n = 1_000_000
    c = np.zeros(n)
    er = np.zeros(n)
    L.ora_sample_kn(E, 99, n, _lib._p(c), _lib._p(er))
    nb = 50
    edges = np.linspace(-1, 1, nb + 1)
    obs, _ = np.histogram(c, edges)
    tot = integrate.quad(lambda x: kn_dsigma_domega(E, x), -1, 1)[0]
    p = np.array([integrate.quad(lambda x: kn_dsigma_domega(E, x), a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) / tot
    chi2 = ((obs - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, nb - 1) > 1e-3
    # Compton kinematics: E'/E = 1 / (1 + k (1 - cos))
    assert np.allclose(er, 1.0 / (1.0 + E / ME * (1.0 - c)), rtol=1e-12)


def test_photoelectric_scaling():
    # Z_eff^3 (Z/A) / E^3 scaling (Z^4/A per atom)
    a = L.ora_mu_rho(0.05, 0, 1)
    assert abs(L.ora_mu_rho(0.1, 0, 1) / a - 0.125) < 1e-12
    ratio = L.ora_mu_rho(0.05, 1, 1) / a
    assert abs(ratio - (13.8 / 7.42) ** 3 * 0.5148 / 0.555087) < 1e-12


def test_pair_threshold():
    assert L.ora_mu_rho(2 * ME * 0.999, 0, 2) == 0.0
    assert L.ora_mu_rho(2 * ME * 1.001, 0, 2) > 0.0
    assert L.ora_mu_rho(6.0, 0, 2) > L.ora_mu_rho(3.0, 0, 2)


def test_compton_mass_attenuation_water_1mev():
    # sigma_KN N_A Z/A for water at 1 MeV: about 0.0707 cm^2/g
    assert abs(L.ora_mu_rho(1.0, 0, 0) / 0.0707 - 1) < 5e-3


# ----------------------------------------------------------- electrons -----
def icru37_collision_stopping(T, I=75e-6, za=ZA_WATER):
    """Unrestricted electron collision stopping power, ICRU Report 37 form,
    no density effect, MeV cm^2/g."""
    tau = T / ME
    b2 = 1 - 1 / (1 + tau) ** 2
    Fm = 1 - b2 + (tau * tau / 8 - (2 * tau + 1) * math.log(2)) / (tau + 1) ** 2
    return (2 * math.pi * RE * RE * ME * NA * za / b2) * (math.log(tau * tau * (tau + 2) / (2 * (I / ME) ** 2)) + Fm)


@pytest.mark.parametrize("T", [0.05, 0.2, 1.0, 3.0, 10.0])
def test_unrestricted_collision_stopping_is_icru37(T):
    assert abs(L.ora_col_stopping(T, T) / icru37_collision_stopping(T) - 1) < 1e-12


def test_collision_stopping_reference_value():
    # water at 1 MeV, no density effect: near the tabulated 1.85 MeV cm^2/g
    assert abs(L.ora_col_stopping(1.0, 1.0) / 1.85 - 1) < 0.02


@pytest.mark.parametrize("T", [0.5, 1.0, 2.5, 6.0])
def test_restricted_stopping_plus_hard_losses_is_unrestricted(T):
    """L(T; T/2) - L(T; W_c) = integral over W_c..T/2 of W dsigma/dW."""
    wc = 0.2
    hard, _ = integrate.quad(lambda W: W * L.ora_moller_dcs(T, W), wc, T / 2, epsrel=1e-11)
    assert abs((L.ora_col_stopping(T, T) - L.ora_col_stopping(T, wc)) / hard - 1) < 1e-8


@pytest.mark.parametrize("T", [0.45, 1.0, 3.0, 6.0])
def test_moller_total_is_integral_of_dcs(T):
    num, _ = integrate.quad(lambda W: L.ora_moller_dcs(T, W), 0.2, T / 2, epsrel=1e-11)
    assert abs(L.ora_moller_sigma(T, 0.2) / num - 1) < 1e-9
    assert L.ora_moller_sigma(0.39, 0.2) == 0.0


@pytest.mark.parametrize("T", [0.6, 2.0, 6.0])
def test_moller_sampler_chi2(T):
    n = 400_000
    eps = np.zeros(n)
    L.ora_sample_moller(T, 0.2, 7, n, _lib._p(eps))
    ec = 0.2 / T
    assert eps.min() >= ec and eps.max() <= 0.5
    edges = np.geomspace(ec, 0.5, 31)
    obs, _ = np.histogram(eps, edges)
    p = np.array([integrate.quad(lambda e: L.ora_moller_dcs(T, e * T), a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    p /= p.sum()
    chi2 = ((obs - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-3


def test_brem_model_consistency():
    # 1/k spectrum: hard cross section = S_rad / T * ln(T / W_cb); soft part S_rad W_cb / T
    for T in (0.5, 2.0, 6.0):
        s = L.ora_rad_stopping(T)
        assert abs(L.ora_brem_sigma(T, 0.2) - s / T * math.log(T / 0.2)) < 1e-15
        tot = L.ora_restricted_stopping(T, 0.2, 0.2)
        assert abs(tot - (L.ora_col_stopping(T, 0.2) + s * 0.2 / T)) < 1e-12
    assert L.ora_brem_sigma(0.19, 0.2) == 0.0


@pytest.mark.parametrize("T", [0.3, 1.0, 4.0, 12.0])
def test_range_is_integral_of_inverse_stopping(T):
    # the restricted stopping power has kinks at T = W_cb and T = 2 W_cc
    f = lambda t: 1.0 / L.ora_restricted_stopping(t, 0.2, 0.2)
    pts = [p for p in (0.2, 0.4) if p < T]
    num, _ = integrate.quad(f, 1e-3, T, epsrel=1e-13, limit=400, points=pts or None)
    assert abs(L.ora_range(T, 0.2, 0.2) / num - 1) < 1e-9
    assert abs(L.ora_range_inv(L.ora_range(T, 0.2, 0.2), 0.2, 0.2) / T - 1) < 1e-12


# ----------------------------------------------------------- positrons -----
def icru37_positron_collision_stopping(T, I=75e-6, za=ZA_WATER):
    """Unrestricted positron collision stopping power, ICRU Report 37 form
    (its F+ function), no density effect, MeV cm^2/g."""
    tau = T / ME
    b2 = 1 - 1 / (1 + tau) ** 2
    Fp = 2 * math.log(2) - (b2 / 12) * (23 + 14 / (tau + 2) + 10 / (tau + 2) ** 2 + 4 / (tau + 2) ** 3)
    return (2 * math.pi * RE * RE * ME * NA * za / b2) * (math.log(tau * tau * (tau + 2) / (2 * (I / ME) ** 2)) + Fp)


def bhabha_dcs_by_hand(T, W):
    """Bhabha cross section per unit energy transfer from its textbook form
    dsigma/deps = 2 pi r_e^2 m c^2 / (beta^2 T) [1/eps^2 - beta^2 (B1/eps - B2
    + B3 eps - B4 eps^2)], gamma = 1 + T/mc^2, y = 1/(gamma + 1), per unit
    mass of water (N_A Z/A), divided by T for per unit W."""
    gam = 1 + T / ME
    b2 = 1 - 1 / gam ** 2
    y = 1 / (gam + 1)
    B1 = 2 - y * y
    B2 = (1 - 2 * y) * (3 + y * y)
    B4 = (1 - 2 * y) ** 3
    B3 = B4 + (1 - 2 * y) ** 2
    e = W / T
    per_eps = 2 * math.pi * RE * RE * ME / (b2 * T) * (1 / e ** 2 - b2 * (B1 / e - B2 + B3 * e - B4 * e * e))
    return per_eps * NA * ZA_WATER / T


@pytest.mark.parametrize("T", [0.05, 0.2, 1.0, 3.0, 10.0])
def test_unrestricted_positron_stopping_is_icru37(T):
    assert abs(L.ora_pos_col_stopping(T, T) / icru37_positron_collision_stopping(T) - 1) < 1e-12
    # above ~1 MeV positrons lose a little less than electrons (ICRU 37)
    if T >= 1.0:
        assert L.ora_pos_col_stopping(T, T) < L.ora_col_stopping(T, T)


@pytest.mark.parametrize("T,W", [(0.5, 0.21), (1.0, 0.3), (1.0, 0.99), (6.0, 0.2), (6.0, 5.5)])
def test_bhabha_dcs_matches_textbook_form(T, W):
    assert L.ora_bhabha_dcs(T, W) == pytest.approx(bhabha_dcs_by_hand(T, W), rel=1e-12)


@pytest.mark.parametrize("T", [0.3, 1.0, 2.5, 6.0])
def test_restricted_positron_stopping_plus_hard_losses_is_unrestricted(T):
    """L+(T; T) - L+(T; W_c) = integral over W_c..T of W dsigma_Bhabha/dW:
    links the restricted stopping power to the hard cross section."""
    wc = 0.2
    hard, _ = integrate.quad(lambda W: W * L.ora_bhabha_dcs(T, W), wc, T, epsrel=1e-11)
    assert abs((L.ora_pos_col_stopping(T, T) - L.ora_pos_col_stopping(T, wc)) / hard - 1) < 1e-8


@pytest.mark.parametrize("T", [0.25, 1.0, 3.0, 6.0])
def test_bhabha_total_is_integral_of_dcs(T):
    num, _ = integrate.quad(lambda W: L.ora_bhabha_dcs(T, W), 0.2, T, epsrel=1e-11)
    assert abs(L.ora_bhabha_sigma(T, 0.2) / num - 1) < 1e-9
    assert L.ora_bhabha_sigma(0.19, 0.2) == 0.0
    # a positron can hand its whole energy to the electron: its hard events
    # start at W_c, below the Moller threshold 2 W_c
    assert L.ora_bhabha_sigma(0.3, 0.2) > 0.0 and L.ora_moller_sigma(0.3, 0.2) == 0.0


def test_bhabha_rejection_bound():
    """The sampler proposes from 1/eps^2 and keeps eps with probability
    eps^2 dsigma/deps / (its Rutherford factor), which must lie in (0, 1]."""
    for T in np.geomspace(0.2, 30.0, 60):
        for e in np.linspace(0.2 / T, 1.0, 200):
            h = bhabha_dcs_by_hand(T, e * T) * (e * T) ** 2 / (2 * math.pi * RE * RE * ME / (1 - 1 / (1 + T / ME) ** 2)
                                                               * NA * ZA_WATER) / T * T
            assert 0.0 < h <= 1.0 + 1e-12, (T, e, h)


@pytest.mark.parametrize("T", [0.5, 2.0, 6.0])
def test_bhabha_sampler_chi2(T):
    n = 400_000
    eps = np.zeros(n)
    L.ora_sample_bhabha(T, 0.2, 9, n, _lib._p(eps))
    ec = 0.2 / T
    assert eps.min() >= ec and eps.max() <= 1.0
    edges = np.geomspace(ec, 1.0, 31)
    obs, _ = np.histogram(eps, edges)
    p = np.array([integrate.quad(lambda e: L.ora_bhabha_dcs(T, e * T), a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    p /= p.sum()
    chi2 = ((obs - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-3


@pytest.mark.parametrize("T", [0.3, 1.0, 4.0, 12.0])
def test_positron_range_is_integral_of_inverse_stopping(T):
    f = lambda t: 1.0 / L.ora_restricted_stopping_pos(t, 0.2, 0.2)
    pts = [p for p in (0.2,) if p < T]
    num, _ = integrate.quad(f, 1e-3, T, epsrel=1e-13, limit=400, points=pts or None)
    assert abs(L.ora_range_pos(T, 0.2, 0.2) / num - 1) < 1e-9
    assert abs(L.ora_range_inv_pos(L.ora_range_pos(T, 0.2, 0.2), 0.2, 0.2) / T - 1) < 1e-12
