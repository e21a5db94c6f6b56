/*
 * CPU oracle of the PSL dose path: photon/electron transport, tally and the
 * physics it needs, in double precision.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: the Philox generator, the physics formulas and the
 * transport loop below are written out here on their own.
 *
 * What the paper fixes and what it does not.  The paper (Sec. 2.3.3) hands
 * particles to "transport as described in Jia et al. (2011)" with atomic dose
 * counters, batch uncertainty (Sec. 2.3.3) and cut-offs of 0.010 MeV for
 * photons and 0.700 MeV for electrons (Sec. 2.6).  It prints no physics.  The
 * physics here is the stated synthetic model of the workload definition:
 * Woodcock photon tracking with Klein-Nishina Compton (Kahn's sampling),
 * Z^4/E^3 photoelectric and a threshold pair fit; class-II condensed-history
 * electrons and positrons with the restricted Bethe collision stopping power
 * (Moller form for electrons, Bhabha form for positrons), hard Moller (e-)
 * or Bhabha (e+) delta rays and hard bremsstrahlung above fixed thresholds
 * and Gaussian (Highland) multiple scattering.  All constants are stated
 * below.
 * Parity of these constants against the paper is unpinned (the paper has
 * none); the tests pin the formulas against closed forms instead.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit seed,
 * counter = (draw/4, stream tag, particle id low, particle id high).
 * uniform = ((r >> 9) + 0.5) * 2^-23: 24 significant bits, so exactly the same
 * value in float and double, strictly inside (0, 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------- constants of the synthetic physics model ---------------- */
#define ME 0.51099895              /* electron rest energy, MeV */
#define RE 2.8179403262e-13        /* classical electron radius, cm */
#define NAV 6.02214076e23          /* Avogadro */
#define PI_D 3.14159265358979323846
#define I_WATER 75.0e-6            /* mean excitation energy of water, MeV */
#define X0_WATER 36.08             /* radiation length of water, g/cm^2 */
#define C_PE 2.0e-8                /* photoelectric: mu/rho = C_PE (Z/A) Zeff^3 / E^3 */
#define C_PP 1.3e-3                /* pair: mu/rho = C_PP (Z/A) Zeff (1 - 2me/E)^3 */
#define T_RANGE_LO 1.0e-3          /* lower end of the range integral, MeV */
#define T_RANGE_HI 30.0            /* upper end of the range table, MeV */
#define N_RANGE 2048               /* range-table nodes (log spaced) */
#define MAX_E_STEPS 100000         /* per-electron step guard */

/* material 0: water-like (air, lung, tissue, water); 1: bone */
static const double MAT_ZA[2] = {0.555087, 0.5148};
static const double MAT_ZEFF[2] = {7.42, 13.8};

/* Philox stream tags */
#define TAG_PARTICLE 0u
#define TAG_OFFSET 1u
#define TAG_CHILD 2u

/* physics switches (tests); 0 in production */
#define F_LOCAL_SECONDARIES 1u  /* secondaries deposit their energy in place */
#define F_FIRST_INTERACTION 2u  /* photons deposit everything at the first real interaction */
#define F_NO_MSC 4u             /* electrons: no multiple-scattering deflection */
#define F_NO_HARD 8u            /* electrons: no hard delta rays or bremsstrahlung */

/* ledger slots */
enum { L_EMITTED = 0, L_ESCAPED, L_DEPOSITED, L_COMPTON, L_PHOTO, L_PAIR, L_ESTEPS, L_ERRORS,
       L_HARD_COLL,    /* hard Moller / Bhabha collisions */
       L_HARD_BREM,    /* hard bremsstrahlung events */
       L_N };

/* ------------------------------- Philox ---------------------------------- */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void ora_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

typedef struct { uint64_t seed, pid; uint32_t draw; } stream_t;

static double uniform(stream_t *s) {
    uint32_t ctr[4] = {s->draw >> 2, TAG_PARTICLE, (uint32_t)s->pid, (uint32_t)(s->pid >> 32)};
    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
    uint32_t out[4];
    philox4x32_10(ctr, key, out);
    uint32_t r = out[s->draw & 3u];
    s->draw++;
    return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Start the next draw at a fresh Philox block.  Every event (a Woodcock step,
 * an interaction, an electron step, a hard event, an annihilation) begins on
 * a block boundary, so the draws of one event come from as few blocks as
 * possible (and a GPU warp refills its blocks together). */
static void align_stream(stream_t *s) { s->draw = (s->draw + 3u) & ~3u; }

/* id of the ordinal-th secondary of particle `parent` (top bit set) */
static uint64_t child_pid(uint64_t seed, uint64_t parent, uint32_t ordinal) {
    uint32_t ctr[4] = {ordinal, TAG_CHILD, (uint32_t)parent, (uint32_t)(parent >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    philox4x32_10(ctr, key, out);
    return ((uint64_t)out[0] | ((uint64_t)out[1] << 32)) | 0x8000000000000000ull;
}

/* ----------------------------- photon physics ---------------------------- */
/* Klein-Nishina total cross section per electron, cm^2 (closed form). */
double ora_kn_sigma(double E) {
    double k = E / ME, a = 1.0 + 2.0 * k, L = log(a);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k);
    double t2 = L / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * PI_D * RE * RE * (t1 + t2 - t3);
}

/* mass attenuation coefficients, cm^2/g; which: 0 Compton, 1 photo, 2 pair, 3 total */
double ora_mu_rho(double E, int mat, int which) {
    double za = MAT_ZA[mat], z = MAT_ZEFF[mat];
    double mc = NAV * za * ora_kn_sigma(E);
    double mpe = C_PE * za * z * z * z / (E * E * E);
    double mpp = 0.0;
    if (E > 2.0 * ME) { double f = 1.0 - 2.0 * ME / E; mpp = C_PP * za * z * f * f * f; }
    switch (which) {
    case 0: return mc;
    case 1: return mpe;
    case 2: return mpp;
    default: return mc + mpe + mpp;
    }
}

/* ---------------------------- electron physics --------------------------- */
static double beta2_of(double T) { double g = 1.0 + T / ME; return 1.0 - 1.0 / (g * g); }

/* Restricted collision stopping power (Moller, no density effect), MeV cm^2/g,
 * for energy transfers below `cut` (MeV).  cut >= T/2 gives the unrestricted
 * Bethe value. Electron density of water-like media. */
double ora_col_stopping(double T, double cut) {
    double tau = T / ME, b2 = beta2_of(T);
    double d = fmin(cut, 0.5 * T) / ME;          /* cut in units of me */
    double iom = I_WATER / ME;
    double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d)
             + (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / ((tau + 1.0) * (tau + 1.0));
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0] / b2;
    return K * (log(2.0 * (tau + 2.0) / (iom * iom)) + F);
}

/* Radiative stopping power fit, MeV cm^2/g: S_rad = (T + me) T / (X0 (T + 2 MeV)). */
double ora_rad_stopping(double T) { return (T + ME) * T / (X0_WATER * (T + 2.0)); }

/* Moller differential cross section per unit energy transfer W, cm^2/(g MeV). */
double ora_moller_dcs(double T, double W) {
    double tau = T / ME, b2 = beta2_of(T), e = W / T;
    double g = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
    double a = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0] / b2;
    return K / (T * T) * (1.0 / (e * e) + 1.0 / ((1.0 - e) * (1.0 - e)) + g - a / (e * (1.0 - e)));
}

/* hard Moller cross section (W from wcc to T/2), cm^2/g */
double ora_moller_sigma(double T, double wcc) {
    if (T <= 2.0 * wcc) return 0.0;
    double tau = T / ME, b2 = beta2_of(T), ec = wcc / T;
    double g = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
    double a = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0] / b2;
    return K / T * (1.0 / ec - 1.0 / (1.0 - ec) + g * (0.5 - ec) - a * log((1.0 - ec) / ec));
}

/* hard bremsstrahlung cross section with a 1/k spectrum above wcb, cm^2/g */
double ora_brem_sigma(double T, double wcb) {
    if (T <= wcb) return 0.0;
    return ora_rad_stopping(T) / T * log(T / wcb);
}

/* total restricted stopping power (soft collisions + soft radiation) */
double ora_restricted_stopping(double T, double wcc, double wcb) {
    return ora_col_stopping(T, wcc) + ora_rad_stopping(T) * fmin(wcb, T) / T;
}

/* ---------------------------- positron physics --------------------------- */
/* Bhabha coefficients of a positron of kinetic energy T: with y = 1/(tau+2),
 * B1 = 2 - y^2, B2 = (1-2y)(3+y^2), B4 = (1-2y)^3, B3 = B4 + (1-2y)^2. */
static void bhabha_b(double T, double b[4]) {
    double y = 1.0 / (T / ME + 2.0), x = 1.0 - 2.0 * y;
    b[0] = 2.0 - y * y;
    b[1] = x * (3.0 + y * y);
    b[3] = x * x * x;
    b[2] = b[3] + x * x;
}

/* Bhabha differential cross section per unit energy W given to the atomic
 * electron (0 < W <= T: the two particles are distinguishable), cm^2/(g MeV):
 * 2 pi r_e^2 m c^2 (N_A Z/A) / T^2 [1/(beta^2 e^2) - B1/e + B2 - B3 e + B4 e^2],
 * e = W/T. */
double ora_bhabha_dcs(double T, double W) {
    double b2 = beta2_of(T), e = W / T, b[4];
    bhabha_b(T, b);
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0];
    return K / (T * T) * (1.0 / (b2 * e * e) - b[0] / e + b[1] - b[2] * e + b[3] * e * e);
}

/* hard Bhabha cross section (W from wcc to T), cm^2/g: the integral of the
 * bracket over e in [ec, 1] */
double ora_bhabha_sigma(double T, double wcc) {
    if (T <= wcc) return 0.0;
    double b2 = beta2_of(T), ec = wcc / T, b[4];
    bhabha_b(T, b);
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0];
    return K / T * ((1.0 / ec - 1.0) / b2 - b[0] * log(1.0 / ec) + b[1] * (1.0 - ec)
                    - b[2] * 0.5 * (1.0 - ec * ec) + b[3] * (1.0 - ec * ec * ec) / 3.0);
}

/* Restricted collision stopping power of a positron (Bhabha, no density
 * effect), MeV cm^2/g, for energy transfers below `cut`; cut >= T gives the
 * unrestricted value.  With d = min(cut, T)/mc^2 and y = 1/(tau+2):
 * K/beta^2 [ln(2 (tau+2) / (I/mc^2)^2) + F+], F+ = ln(tau d) - (beta^2/tau)
 * [tau + 2d - 3 d^2 y/2 - (d - d^3/3) y^2 - (d^2/2 - tau d^3/3 + d^4/4) y^3]. */
double ora_pos_col_stopping(double T, double cut) {
    double tau = T / ME, b2 = beta2_of(T), d = fmin(cut, T) / ME, y = 1.0 / (tau + 2.0);
    double iom = I_WATER / ME;
    double F = log(tau * d) - (b2 / tau) * (tau + 2.0 * d - 1.5 * d * d * y - (d - d * d * d / 3.0) * y * y
                                             - (0.5 * d * d - tau * d * d * d / 3.0 + 0.25 * d * d * d * d) * y * y * y);
    double K = 2.0 * PI_D * RE * RE * ME * NAV * MAT_ZA[0] / b2;
    return K * (log(2.0 * (tau + 2.0) / (iom * iom)) + F);
}

double ora_restricted_stopping_pos(double T, double wcc, double wcb) {
    return ora_pos_col_stopping(T, wcc) + ora_rad_stopping(T) * fmin(wcb, T) / T;
}

/* restricted stopping power of a species (0 electron, 1 positron) */
static double restricted_stopping(int pos, double T, double wcc, double wcb) {
    return pos ? ora_restricted_stopping_pos(T, wcc, wcb) : ora_restricted_stopping(T, wcc, wcb);
}

/* hard collision (delta-ray) cross section of a species, cm^2/g */
static double hard_collision_sigma(int pos, double T, double wcc) {
    return pos ? ora_bhabha_sigma(T, wcc) : ora_moller_sigma(T, wcc);
}

/* ----------------------- CSDA range with restricted S --------------------- */
static double gl_x[16], gl_w[16];
static double rt_T[N_RANGE], rt_R[2][N_RANGE];    /* [species][node]: 0 electron, 1 positron */
static double rt_wcc = -1.0, rt_wcb = -1.0;

static void gauss_legendre16(void) {
    /* nodes and weights on [-1, 1] by Newton iteration on P_16 */
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double x = cos(PI_D * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static double int_inv_s(int pos, double a, double b, double wcc, double wcb) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < 16; ++i) s += gl_w[i] / restricted_stopping(pos, m + h * gl_x[i], wcc, wcb);
    return s * h;
}

static void range_setup(double wcc, double wcb) {
    if (rt_wcc == wcc && rt_wcb == wcb) return;
    gauss_legendre16();
    double lr = log(T_RANGE_HI / T_RANGE_LO);
    for (int i = 0; i < N_RANGE; ++i) rt_T[i] = T_RANGE_LO * exp(lr * i / (N_RANGE - 1));
    for (int p = 0; p < 2; ++p) {
        rt_R[p][0] = 0.0;
        for (int i = 1; i < N_RANGE; ++i) rt_R[p][i] = rt_R[p][i - 1] + int_inv_s(p, rt_T[i - 1], rt_T[i], wcc, wcb);
    }
    rt_wcc = wcc; rt_wcb = wcb;
}

/* R(T) = integral from T_RANGE_LO to T of dT'/S_restricted of the species, g/cm^2 */
static double range_of(int pos, double T, double wcc, double wcb) {
    int lo = 0, hi = N_RANGE - 1;
    if (T <= rt_T[0]) return 0.0;
    while (hi - lo > 1) { int mid = (lo + hi) / 2; if (rt_T[mid] <= T) lo = mid; else hi = mid; }
    return rt_R[pos][lo] + int_inv_s(pos, rt_T[lo], T, wcc, wcb);
}

/* inverse of range_of by Newton's method (dR/dT = 1/S) */
static double range_inv(int pos, double r, double wcc, double wcb) {
    if (r <= 0.0) return T_RANGE_LO;
    const double *R = rt_R[pos];
    int lo = 0, hi = N_RANGE - 1;
    while (hi - lo > 1) { int mid = (lo + hi) / 2; if (R[mid] <= r) lo = mid; else hi = mid; }
    double a = rt_T[lo], b = rt_T[hi];
    double T = a + (b - a) * (r - R[lo]) / (R[hi] - R[lo]);
    for (int it = 0; it < 60; ++it) {
        double f = range_of(pos, T, wcc, wcb) - r;
        double Tn = T - f * restricted_stopping(pos, T, wcc, wcb);
        if (Tn < a) Tn = a;
        if (Tn > b) Tn = b;
        if (fabs(Tn - T) <= 1e-15 * T) { T = Tn; break; }
        T = Tn;
    }
    return T;
}

double ora_range(double T, double wcc, double wcb) { range_setup(wcc, wcb); return range_of(0, T, wcc, wcb); }
double ora_range_inv(double r, double wcc, double wcb) { range_setup(wcc, wcb); return range_inv(0, r, wcc, wcb); }
double ora_range_pos(double T, double wcc, double wcb) { range_setup(wcc, wcb); return range_of(1, T, wcc, wcb); }
double ora_range_inv_pos(double r, double wcc, double wcb) { range_setup(wcc, wcb); return range_inv(1, r, wcc, wcb); }

/* ------------------------------- sampling -------------------------------- */
/* Kahn's rejection method for the Klein-Nishina distribution.  Returns
 * x = E/E' (> 1); cos(theta) = 1 - (x - 1)/k. */
static double sample_kahn(double E, stream_t *s) {
    double k = E / ME;
    for (;;) {
        double r1 = uniform(s), r2 = uniform(s), r3 = uniform(s);
        if (r1 <= (1.0 + 2.0 * k) / (9.0 + 2.0 * k)) {
            double x = 1.0 + 2.0 * k * r2;
            if (r3 <= 4.0 * (1.0 / x - 1.0 / (x * x))) return x;
        } else {
            double x = (1.0 + 2.0 * k) / (1.0 + 2.0 * k * r2);
            double c = 1.0 - (x - 1.0) / k;
            if (r3 <= 0.5 * (c * c + 1.0 / x)) return x;
        }
    }
}

/* Moller energy-transfer fraction eps in [wcc/T, 1/2].  The bracket of the
 * cross section times eps^2 is bounded by 1 + 5 eps^2, so eps is proposed
 * from the density 1/eps^2 + 5 (a mixture of 1/eps^2 and a uniform part,
 * picked by their integrals) and accepted with probability bracket/(1+5eps^2). */
static double sample_moller(double T, double wcc, stream_t *s) {
    double tau = T / ME, ec = wcc / T;
    double g = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
    double a = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    double w1 = 1.0 / ec - 2.0, w2 = 5.0 * (0.5 - ec);
    for (;;) {
        double r1 = uniform(s), r2 = uniform(s), r3 = uniform(s);
        double e;
        if (r1 * (w1 + w2) < w1) e = ec / (1.0 - r2 * (1.0 - 2.0 * ec));
        else e = ec + r2 * (0.5 - ec);
        double q = e / (1.0 - e);
        double f = 1.0 + q * q + g * e * e - a * q;
        if (r3 * (1.0 + 5.0 * e * e) <= f) return e;
    }
}

void ora_sample_kn(double E, uint64_t seed, int64_t n, double *cos_out, double *eratio_out) {
    double k = E / ME;
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        double x = sample_kahn(E, &s);
        cos_out[i] = 1.0 - (x - 1.0) / k;
        if (eratio_out) eratio_out[i] = 1.0 / x;
    }
}

void ora_sample_moller(double T, double wcc, uint64_t seed, int64_t n, double *eps_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        eps_out[i] = sample_moller(T, wcc, &s);
    }
}

/* Bhabha energy-transfer fraction e in [wcc/T, 1] (the atomic electron
 * gets e T).  The cross section is (1/e^2) h(e) with
 * h(e) = 1 - beta^2 e (B1 - e (B2 - e (B3 - e B4))), and 0 < h <= 1 on
 * (0, 1] (checked by the tests), so e is proposed from the density 1/e^2 on
 * [ec, 1] and accepted with probability h(e). */
static double sample_bhabha(double T, double wcc, stream_t *s) {
    double ec = wcc / T, b2 = beta2_of(T), b[4];
    bhabha_b(T, b);
    for (;;) {
        double r1 = uniform(s), r2 = uniform(s);
        double e = ec / (1.0 - r1 * (1.0 - ec));
        double h = 1.0 - b2 * e * (b[0] - e * (b[1] - e * (b[2] - e * b[3])));
        if (r2 <= h) return e;
    }
}

void ora_sample_bhabha(double T, double wcc, uint64_t seed, int64_t n, double *eps_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        eps_out[i] = sample_bhabha(T, wcc, &s);
    }
}

/* Highland's characteristic multiple-scattering angle (radians) of a step of
 * s cm at density rho: theta0 = 13.6 MeV / (beta c p) sqrt(t) (1 + 0.038 ln t),
 * t = s rho / X0 (the water radiation length scaled by density), with
 * beta c p = T (T + 2 m c^2) / (T + m c^2); 0 where the bracket is not positive. */
double ora_highland(double T, double s, double rho) {
    double x0 = X0_WATER / rho, t = s / x0;
    if (t <= 0.0) return 0.0;
    double bcp = T * (T + 2.0 * ME) / (T + ME);
    double f = 1.0 + 0.038 * log(t);
    if (f <= 0.0) return 0.0;
    return 13.6 / bcp * sqrt(t) * f;
}

/* The multiple-scattering deflection of a step: polar angle theta =
 * theta0 sqrt(-2 ln u) (the space angle of a two-dimensional Gaussian of
 * width theta0 per projected plane: Rayleigh distributed), azimuth 2 pi u'. */
static void sample_msc(double th0, stream_t *s, double *theta, double *phi) {
    *theta = th0 * sqrt(-2.0 * log(uniform(s)));
    *phi = 2.0 * PI_D * uniform(s);
}

void ora_sample_msc(double th0, uint64_t seed, int64_t n, double *theta_out, double *phi_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        sample_msc(th0, &s, theta_out + i, phi_out + i);
    }
}

/* Energy of a hard bremsstrahlung photon: the 1/k spectrum on [wcb, T],
 * k = wcb (T/wcb)^u. */
static double sample_brem_photon(double T, double wcb, stream_t *s) {
    return wcb * exp(uniform(s) * log(T / wcb));
}

void ora_sample_brem(double T, double wcb, uint64_t seed, int64_t n, double *k_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        k_out[i] = sample_brem_photon(T, wcb, &s);
    }
}

/* Pair production: the kinetic energy E - 2 m c^2 split uniformly between
 * the electron (t1) and the positron (t2). */
static void sample_pair_split(double E, stream_t *s, double *t1, double *t2) {
    double avail = E - 2.0 * ME;
    *t1 = uniform(s) * avail;
    *t2 = avail - *t1;
}

void ora_sample_pair(double E, uint64_t seed, int64_t n, double *t1_out, double *t2_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        sample_pair_split(E, &s, t1_out + i, t2_out + i);
    }
}

/* Annihilation at rest: the first photon's direction uniform on the sphere
 * (cos theta = 2u - 1, azimuth 2 pi u'); the second goes the opposite way. */
static void sample_annihilation(stream_t *s, double a[3]) {
    double cth = 2.0 * uniform(s) - 1.0, phi = 2.0 * PI_D * uniform(s);
    double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    a[0] = sth * cos(phi); a[1] = sth * sin(phi); a[2] = cth;
}

void ora_sample_annihilation(uint64_t seed, int64_t n, double *d1_out, double *d2_out) {
    for (int64_t i = 0; i < n; ++i) {
        stream_t s = {seed, (uint64_t)i, 0};
        double a[3];
        sample_annihilation(&s, a);
        for (int k = 0; k < 3; ++k) { d1_out[3 * i + k] = a[k]; d2_out[3 * i + k] = -a[k]; }
    }
}

/* Rotate unit direction d by polar cosine c and azimuth phi.  The azimuth
 * is measured from the plane through d and the z axis:
 *   d' = c d + sin(theta) (cos(phi) e1 + sin(phi) e2),
 *   e1 = (u w, v w, -t) / t,  e2 = (-v, u, 0) / t,  t = sqrt(u^2 + v^2),
 * an orthonormal pair perpendicular to d, so d.d' = c exactly.  Only a
 * direction on the z axis itself (t^2 <= 1e-30) takes the fixed pair
 * e1 = (1, 0, 0), e2 = (0, 1, 0). */
static void rotate_dir(double d[3], double c, double phi) {
    double st = sqrt(fmax(0.0, 1.0 - c * c)), cp = cos(phi), sp = sin(phi);
    double u = d[0], v = d[1], w = d[2], nu, nv, nw;
    double t2 = u * u + v * v;
    if (t2 <= 1e-30) {
        nu = st * cp; nv = st * sp; nw = (w > 0 ? c : -c);
    } else {
        double t = sqrt(t2);
        nu = u * c + st * (u * w * cp - v * sp) / t;
        nv = v * c + st * (v * w * cp + u * sp) / t;
        nw = w * c - st * cp * t;
    }
    double n = sqrt(nu * nu + nv * nv + nw * nw);
    d[0] = nu / n; d[1] = nv / n; d[2] = nw / n;
}

void ora_rotate(int64_t n, const double *d_in, const double *c, const double *phi, double *d_out) {
    for (int64_t i = 0; i < n; ++i) {
        double d[3] = {d_in[3 * i], d_in[3 * i + 1], d_in[3 * i + 2]};
        rotate_dir(d, c[i], phi[i]);
        for (int k = 0; k < 3; ++k) d_out[3 * i + k] = d[k];
    }
}

/* ------------------------------- transport ------------------------------- */
typedef struct {
    int nx, ny, nz;
    double vx, vy, vz;
    const uint8_t *mat;
    const float *rho;
    double rho_max[2];           /* largest density per material (majorant) */
    uint64_t seed;
    uint32_t flags;
    double pcut, ecut, wcc, wcb;
    int64_t *tally;              /* [nvox], added to */
    int64_t *hist_dep, *hist_esc;/* per primary (optional) */
    int32_t *hist_events;
    double *hist_path;
} ctx_t;

typedef struct { int type; double p[3], d[3], E, wt; uint64_t pid; } part_t;  /* type 0 photon, 1 e-, 2 e+ */

typedef struct { part_t *a; int n, cap; } pstack_t;

static void push(pstack_t *s, const part_t *p) {
    if (s->n == s->cap) { s->cap = s->cap ? 2 * s->cap : 64; s->a = (part_t *)realloc(s->a, sizeof(part_t) * s->cap); }
    s->a[s->n++] = *p;
}

typedef struct { int64_t ledger[L_N]; int64_t dep, esc; int32_t events; double path; } acc_t;

static int64_t fixed_point(double mev_wt) { return llrint(mev_wt * 4294967296.0); }

static void deposit(const ctx_t *c, acc_t *a, int64_t iv, double e, double wt) {
    int64_t q = fixed_point(e * wt);
    if (q == 0) return;
    __atomic_fetch_add(&c->tally[iv], q, __ATOMIC_RELAXED);
    a->ledger[L_DEPOSITED] += q;
    a->dep += q;
}

static void escape(acc_t *a, double e, double wt) {
    int64_t q = fixed_point(e * wt);
    a->ledger[L_ESCAPED] += q;
    a->esc += q;
}

static int voxel_of(const ctx_t *c, const double p[3], int64_t *iv) {
    double fx = floor(p[0] / c->vx), fy = floor(p[1] / c->vy), fz = floor(p[2] / c->vz);
    if (fx < 0 || fy < 0 || fz < 0 || fx >= c->nx || fy >= c->ny || fz >= c->nz) return 0;
    *iv = ((int64_t)fz * c->ny + (int64_t)fy) * c->nx + (int64_t)fx;
    return 1;
}

static double mu_max_of(const ctx_t *c, double E) {
    double m0 = c->rho_max[0] * ora_mu_rho(E, 0, 3), m1 = c->rho_max[1] * ora_mu_rho(E, 1, 3);
    return m0 > m1 ? m0 : m1;
}

static void annihilate(const ctx_t *c, stream_t *s, uint32_t *nchild, uint64_t pid, const double p[3],
                       double wt, pstack_t *st) {
    align_stream(s);
    double a[3];
    sample_annihilation(s, a);
    for (int k = 0; k < 2; ++k) {
        part_t g = {0, {p[0], p[1], p[2]}, {k ? -a[0] : a[0], k ? -a[1] : a[1], k ? -a[2] : a[2]}, ME, wt,
                    child_pid(c->seed, pid, (*nchild)++)};
        push(st, &g);
    }
}

/* a new charged secondary: transported, or deposited in place */
static void emit_charged(const ctx_t *c, acc_t *a, int type, double T, const double p[3], const double d[3],
                         double wt, int64_t iv, uint64_t pid, uint32_t *nchild, stream_t *s, pstack_t *st) {
    if (T > c->ecut && !(c->flags & F_LOCAL_SECONDARIES)) {
        part_t e = {type, {p[0], p[1], p[2]}, {d[0], d[1], d[2]}, T, wt, child_pid(c->seed, pid, (*nchild)++)};
        push(st, &e);
        return;
    }
    deposit(c, a, iv, T, wt);
    if (type == 2) {
        if (c->flags & F_LOCAL_SECONDARIES) deposit(c, a, iv, 2.0 * ME, wt);
        else annihilate(c, s, nchild, pid, p, wt, st);
    }
}

static void photon(const ctx_t *c, acc_t *a, part_t *g, pstack_t *st) {
    stream_t s = {c->seed, g->pid, 0};
    uint32_t nchild = 0;
    double E = g->E, wt = g->wt, p[3] = {g->p[0], g->p[1], g->p[2]}, d[3] = {g->d[0], g->d[1], g->d[2]};
    for (;;) {
        double mumax = mu_max_of(c, E);
        align_stream(&s);                                  /* Woodcock step: step, virtual, channel */
        double step = -log(uniform(&s)) / mumax;
        for (int k = 0; k < 3; ++k) p[k] += step * d[k];
        int64_t iv;
        if (!voxel_of(c, p, &iv)) { escape(a, E, wt); return; }
        int m = c->mat[iv];
        double rho = c->rho[iv];
        double mc = rho * ora_mu_rho(E, m, 0), mpe = rho * ora_mu_rho(E, m, 1), mpp = rho * ora_mu_rho(E, m, 2);
        double mu = mc + mpe + mpp;
        if (mu > mumax * (1.0 + 1e-12)) a->ledger[L_ERRORS]++;
        if (uniform(&s) * mumax >= mu) continue;          /* virtual (delta) interaction */
        a->events++;
        double r = uniform(&s) * mu;
        align_stream(&s);                                  /* the interaction's draws */
        if (r < mc) {                                      /* Compton */
            a->ledger[L_COMPTON]++;
            if (c->flags & F_FIRST_INTERACTION) { deposit(c, a, iv, E, wt); return; }
            double k = E / ME, x = sample_kahn(E, &s);
            double cth = 1.0 - (x - 1.0) / k;
            if (cth < -1.0) cth = -1.0;
            if (cth > 1.0) cth = 1.0;
            double Ep = E / x, phi = 2.0 * PI_D * uniform(&s);
            double dn[3] = {d[0], d[1], d[2]};
            rotate_dir(dn, cth, phi);
            double Te = E - Ep;
            double de[3] = {E * d[0] - Ep * dn[0], E * d[1] - Ep * dn[1], E * d[2] - Ep * dn[2]};
            double nn = sqrt(de[0] * de[0] + de[1] * de[1] + de[2] * de[2]);
            if (nn > 0) { de[0] /= nn; de[1] /= nn; de[2] /= nn; } else { de[0] = d[0]; de[1] = d[1]; de[2] = d[2]; }
            emit_charged(c, a, 1, Te, p, de, wt, iv, g->pid, &nchild, &s, st);
            E = Ep; d[0] = dn[0]; d[1] = dn[1]; d[2] = dn[2];
            if (E < c->pcut) { deposit(c, a, iv, E, wt); return; }
        } else if (r < mc + mpe) {                         /* photoelectric */
            a->ledger[L_PHOTO]++;
            if (c->flags & F_FIRST_INTERACTION) { deposit(c, a, iv, E, wt); return; }
            emit_charged(c, a, 1, E, p, d, wt, iv, g->pid, &nchild, &s, st);
            return;
        } else {                                           /* pair */
            a->ledger[L_PAIR]++;
            if (c->flags & F_FIRST_INTERACTION) { deposit(c, a, iv, E, wt); return; }
            double T1, T2;
            sample_pair_split(E, &s, &T1, &T2);
            emit_charged(c, a, 1, T1, p, d, wt, iv, g->pid, &nchild, &s, st);
            emit_charged(c, a, 2, T2, p, d, wt, iv, g->pid, &nchild, &s, st);
            return;
        }
    }
}

static void electron(const ctx_t *c, acc_t *a, part_t *e, pstack_t *st) {
    stream_t s = {c->seed, e->pid, 0};
    uint32_t nchild = 0;
    int pos = (e->type == 2);
    double T = e->E, wt = e->wt, p[3] = {e->p[0], e->p[1], e->p[2]}, d[3] = {e->d[0], e->d[1], e->d[2]};
    int ix[3];
    int n[3] = {c->nx, c->ny, c->nz};
    double v[3] = {c->vx, c->vy, c->vz};
    for (int k = 0; k < 3; ++k) {
        double f = floor(p[k] / v[k]);
        ix[k] = f < 0 ? 0 : (f >= n[k] ? n[k] - 1 : (int)f);
    }
    int hard_on = !(c->flags & F_NO_HARD);
    double nlam = -1.0;             /* mean free paths to the next hard event; < 0: draw at the next step */
    double R = range_of(pos, T, c->wcc, c->wcb);
    int steps = 0;
    for (;;) {
        int64_t iv = ((int64_t)ix[2] * c->ny + ix[1]) * c->nx + ix[0];
        if (T <= c->ecut || ++steps > MAX_E_STEPS) {
            if (steps > MAX_E_STEPS) a->ledger[L_ERRORS]++;
            deposit(c, a, iv, T, wt);
            if (pos) {
                if (c->flags & F_LOCAL_SECONDARIES) deposit(c, a, iv, 2.0 * ME, wt);
                else annihilate(c, &s, &nchild, e->pid, p, wt, st);
            }
            return;
        }
        a->ledger[L_ESTEPS]++;
        a->events++;
        align_stream(&s);                                  /* the step's draws */
        if (nlam < 0.0) nlam = -log(uniform(&s));          /* a new mean free path count */
        double rho = c->rho[iv];
        double sig = hard_on ? rho * (hard_collision_sigma(pos, T, c->wcc) + ora_brem_sigma(T, c->wcb)) : 0.0;
        double s_hard = sig > 0.0 ? nlam / sig : INFINITY;
        /* distance to the voxel boundary */
        double s_bound = INFINITY;
        int axis = -1, cross = 0;
        for (int k = 0; k < 3; ++k) {
            double t;
            if (d[k] > 0) t = ((ix[k] + 1) * v[k] - p[k]) / d[k];
            else if (d[k] < 0) t = (ix[k] * v[k] - p[k]) / d[k];
            else continue;
            if (t < 0) t = 0;
            if (t < s_bound) { s_bound = t; axis = k; cross = d[k] > 0 ? 1 : -1; }
        }
        double Tlim = fmax(0.9 * T, c->ecut);
        double Rlim = range_of(pos, Tlim, c->wcc, c->wcb);
        double s_max = (R - Rlim) / rho;
        int which;                                          /* 0 hard, 1 boundary, 2 energy-loss limit */
        double step;
        if (s_hard <= s_bound && s_hard <= s_max) { which = 0; step = s_hard; }
        else if (s_bound <= s_max) { which = 1; step = s_bound; }
        else { which = 2; step = s_max; }
        double Tend, Rend;
        if (which == 2) { Tend = Tlim; Rend = Rlim; }
        else { Rend = R - rho * step; Tend = range_inv(pos, Rend, c->wcc, c->wcb); if (Tend < Tlim) Tend = Tlim; }
        double th0 = ora_highland(T, step, rho);
        deposit(c, a, iv, T - Tend, wt);
        a->path += step;
        T = Tend; R = Rend;
        for (int k = 0; k < 3; ++k) p[k] += step * d[k];
        nlam -= step * sig;
        if (!(c->flags & F_NO_MSC) && step > 0.0) {
            double th, phi;
            sample_msc(th0, &s, &th, &phi);
            rotate_dir(d, cos(th), phi);
        }
        if (which == 1) {
            int k = axis;
            p[k] = (cross > 0 ? (ix[k] + 1) : ix[k]) * v[k];
            ix[k] += cross;
            if (ix[k] < 0 || ix[k] >= n[k]) {
                escape(a, T + (pos ? 2.0 * ME : 0.0), wt);
                return;
            }
        } else if (which == 0) {
            double sm = hard_collision_sigma(pos, T, c->wcc), sb = ora_brem_sigma(T, c->wcb);
            align_stream(&s);                              /* the hard event's draws */
            double r = uniform(&s) * (sm + sb);
            if (sm + sb > 0.0) {
                if (r < sm) {                                /* hard Moller (e-) or Bhabha (e+) */
                    a->ledger[L_HARD_COLL]++;
                    double eps = pos ? sample_bhabha(T, c->wcc, &s) : sample_moller(T, c->wcc, &s);
                    double W = eps * T, Tp = T - W;           /* W to the atomic electron */
                    double cp = sqrt(Tp * (T + 2.0 * ME) / (T * (Tp + 2.0 * ME)));
                    double cd = sqrt(W * (T + 2.0 * ME) / (T * (W + 2.0 * ME)));
                    double phi = 2.0 * PI_D * uniform(&s);
                    double dd[3] = {d[0], d[1], d[2]};
                    rotate_dir(dd, cd, phi + PI_D);
                    rotate_dir(d, cp, phi);
                    emit_charged(c, a, 1, W, p, dd, wt, iv, e->pid, &nchild, &s, st);
                    T = Tp;
                } else {                                     /* hard bremsstrahlung */
                    a->ledger[L_HARD_BREM]++;
                    double kph = sample_brem_photon(T, c->wcb, &s);
                    if (c->flags & F_LOCAL_SECONDARIES) deposit(c, a, iv, kph, wt);
                    else {
                        part_t g = {0, {p[0], p[1], p[2]}, {d[0], d[1], d[2]}, kph, wt, child_pid(c->seed, e->pid, nchild++)};
                        push(st, &g);
                    }
                    T -= kph;
                }
                R = range_of(pos, T, c->wcc, c->wcb);
            }
            nlam = -1.0;                                   /* drawn at the next step */
        }
    }
}

/*
 * Transport n primaries (phantom-local coordinates, cm) and add their dose to
 * `tally` (int64 fixed point, 2^-32 MeV per unit weight).  ledger[10] is added
 * to (escaped, deposited, interaction and step counts, errors, hard
 * collision and hard bremsstrahlung events); the emitted
 * slot belongs to the source stage.  Per-primary sums over the whole
 * secondary tree (deposited and escaped fixed point, events, electron path
 * length in cm) are optional outputs.
 */
int ora_transport(int64_t n, const int32_t *type, const double *pos, const double *dir, const double *E,
                  const double *wt, const uint64_t *pid,
                  int nx, int ny, int nz, double vx, double vy, double vz,
                  const uint8_t *mat, const float *rho,
                  uint64_t seed, uint32_t flags, double pcut, double ecut, double wcc, double wcb,
                  int64_t *tally, int64_t *ledger, int64_t *hist_dep, int64_t *hist_esc, int32_t *hist_events,
                  double *hist_path, int nthreads) {
    ctx_t c;
    c.nx = nx; c.ny = ny; c.nz = nz; c.vx = vx; c.vy = vy; c.vz = vz;
    c.mat = mat; c.rho = rho; c.seed = seed; c.flags = flags;
    c.pcut = pcut; c.ecut = ecut; c.wcc = wcc; c.wcb = wcb;
    c.tally = tally; c.hist_dep = hist_dep; c.hist_esc = hist_esc; c.hist_events = hist_events; c.hist_path = hist_path;
    c.rho_max[0] = c.rho_max[1] = 0.0;
    int64_t nvox = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < nvox; ++i) {
        int m = mat[i];
        if (rho[i] > c.rho_max[m]) c.rho_max[m] = rho[i];
    }
    range_setup(wcc, wcb);
    int64_t tot[L_N];
    memset(tot, 0, sizeof(tot));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        int64_t loc[L_N];
        memset(loc, 0, sizeof(loc));
        pstack_t st = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            acc_t a;
            memset(&a, 0, sizeof(a));
            part_t p0 = {type[i], {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]},
                         {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]}, E[i], wt[i], pid[i]};
            st.n = 0;
            push(&st, &p0);
            while (st.n > 0) {
                part_t q = st.a[--st.n];
                if (q.type == 0) photon(&c, &a, &q, &st);
                else electron(&c, &a, &q, &st);
            }
            for (int k = 0; k < L_N; ++k) loc[k] += a.ledger[k];
            if (hist_dep) hist_dep[i] = a.dep;
            if (hist_esc) hist_esc[i] = a.esc;
            if (hist_events) hist_events[i] = a.events;
            if (hist_path) hist_path[i] = a.path;
        }
        free(st.a);
        for (int k = 0; k < L_N; ++k) __atomic_fetch_add(&tot[k], loc[k], __ATOMIC_RELAXED);
    }
    for (int k = 0; k < L_N; ++k) ledger[k] += tot[k];
    return 0;
}

