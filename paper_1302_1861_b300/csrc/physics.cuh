// Physics of the synthetic transport model, evaluated in double precision on
// the device to fill float32 tables (one entry per log-spaced energy node).
//
// Photons (mass attenuation, cm^2/g):
//   Compton       N_A (Z/A) sigma_KN(E), Klein-Nishina total cross section
//   photoelectric C_PE (Z/A) Zeff^3 / E^3            (Z^4 / (A E^3) per atom)
//   pair          C_PP (Z/A) Zeff (1 - 2 m c^2 / E)^3,  E > 2 m c^2
// Electrons and positrons (water-like electron density for every medium,
// density scaled): restricted collision stopping power (energy transfers
// below W_cc, mean excitation energy 75 eV, no density effect; Moller form
// for electrons, Bhabha form for positrons), radiative stopping
// (T + m) T / (X0 (T + 2 MeV)) with a 1/k spectrum, of which the part below
// W_cb is continuous; hard Moller (e-) or Bhabha (e+) and bremsstrahlung
// cross sections above W_cc and W_cb.
#pragma once

#define PH_ME 0.51099895
#define PH_RE 2.8179403262e-13
#define PH_NA 6.02214076e23
#define PH_PI 3.14159265358979323846
#define PH_I_WATER 75.0e-6
#define PH_X0 36.08
#define PH_C_PE 2.0e-8
#define PH_C_PP 1.3e-3
#define PH_ZA_WATER 0.555087

// material 0 water-like, 1 bone
__host__ __device__ inline double mat_za(int m) { return m ? 0.5148 : 0.555087; }
__host__ __device__ inline double mat_zeff(int m) { return m ? 13.8 : 7.42; }

__device__ inline double ph_kn_sigma(double E) {
    const double k = E / PH_ME, a = 1.0 + 2.0 * k, L = log(a);
    return 2.0 * PH_PI * PH_RE * PH_RE *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k) + L / (2.0 * k) - (1.0 + 3.0 * k) / (a * a));
}

__device__ inline void ph_mu_rho(double E, int m, double &mc, double &mpe, double &mpp) {
    const double za = mat_za(m), z = mat_zeff(m);
    mc = PH_NA * za * ph_kn_sigma(E);
    mpe = PH_C_PE * za * z * z * z / (E * E * E);
    mpp = 0.0;
    if (E > 2.0 * PH_ME) {
        const double f = 1.0 - 2.0 * PH_ME / E;
        mpp = PH_C_PP * za * z * f * f * f;
    }
}

__device__ inline double el_beta2(double T) { const double g = 1.0 + T / PH_ME; return 1.0 - 1.0 / (g * g); }
__device__ inline double el_K(double T) { return 2.0 * PH_PI * PH_RE * PH_RE * PH_ME * PH_NA * PH_ZA_WATER / el_beta2(T); }

__device__ inline double el_col_restricted(double T, double cut) {
    const double tau = T / PH_ME, b2 = el_beta2(T), d = fmin(cut, 0.5 * T) / PH_ME, iom = PH_I_WATER / PH_ME;
    const double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d) +
                     (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / ((tau + 1.0) * (tau + 1.0));
    return el_K(T) * (log(2.0 * (tau + 2.0) / (iom * iom)) + F);
}

__device__ inline double el_rad(double T) { return (T + PH_ME) * T / (PH_X0 * (T + 2.0)); }

__device__ inline double el_moller_sigma(double T, double wcc) {
    if (T <= 2.0 * wcc) return 0.0;
    const double tau = T / PH_ME, ec = wcc / T, g = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
    const double a = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    return el_K(T) / T * (1.0 / ec - 1.0 / (1.0 - ec) + g * (0.5 - ec) - a * log((1.0 - ec) / ec));
}

__device__ inline double el_brem_sigma(double T, double wcb) { return T <= wcb ? 0.0 : el_rad(T) / T * log(T / wcb); }

__device__ inline double el_stop_restricted(double T, double wcc, double wcb) {
    return el_col_restricted(T, wcc) + el_rad(T) * fmin(wcb, T) / T;
}

// Positrons.  Bhabha scattering on an atomic electron that takes the energy
// W = x T, x in (0, 1] (the two are distinguishable): per unit x,
//   2 pi r_e^2 m c^2 n / T * (1/(beta^2 x^2) - B1/x + B2 - B3 x + B4 x^2),
// y = 1/(tau + 2), B1 = 2 - y^2, B2 = (1 - 2y)(3 + y^2), B4 = (1 - 2y)^3,
// B3 = B4 + (1 - 2y)^2.
struct BhabhaB { double b1, b2, b3, b4; };

__host__ __device__ inline BhabhaB bhabha_coeffs(double T) {
    const double y = 1.0 / (T / PH_ME + 2.0), q = 1.0 - 2.0 * y, q2 = q * q;
    BhabhaB c;
    c.b1 = 2.0 - y * y;
    c.b2 = q * (3.0 + y * y);
    c.b4 = q2 * q;
    c.b3 = c.b4 + q2;
    return c;
}

// hard Bhabha cross section (W from wcc to T), cm^2/g
__device__ inline double pos_bhabha_sigma(double T, double wcc) {
    if (T <= wcc) return 0.0;
    const BhabhaB c = bhabha_coeffs(T);
    const double x0 = wcc / T, b2 = el_beta2(T);
    const double k = 2.0 * PH_PI * PH_RE * PH_RE * PH_ME * PH_NA * PH_ZA_WATER / T;
    const double poly = (1.0 - x0) * (c.b2 - 0.5 * c.b3 * (1.0 + x0) + c.b4 * (1.0 + x0 + x0 * x0) / 3.0);
    return k * ((1.0 - x0) / (b2 * x0) - c.b1 * log(1.0 / x0) + poly);
}

// restricted collision stopping power of a positron (transfers below cut)
__device__ inline double pos_col_restricted(double T, double cut) {
    const double tau = T / PH_ME, b2 = el_beta2(T), d = fmin(cut, T) / PH_ME, y = 1.0 / (tau + 2.0);
    const double iom = PH_I_WATER / PH_ME, d2 = d * d, d3 = d2 * d;
    const double brk = tau + 2.0 * d - 1.5 * d2 * y - (d - d3 / 3.0) * y * y - (0.5 * d2 - tau * d3 / 3.0 + 0.25 * d2 * d2) * y * y * y;
    return el_K(T) * (log(2.0 * (tau + 2.0) / (iom * iom)) + log(tau * d) - b2 / tau * brk);
}

__device__ inline double pos_stop_restricted(double T, double wcc, double wcb) {
    return pos_col_restricted(T, wcc) + el_rad(T) * fmin(wcb, T) / T;
}

// restricted stopping power of species sp (0 electron, 1 positron)
__device__ inline double stop_restricted(int sp, double T, double wcc, double wcb) {
    return sp ? pos_stop_restricted(T, wcc, wcb) : el_stop_restricted(T, wcc, wcb);
}
