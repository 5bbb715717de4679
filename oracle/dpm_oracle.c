/*
 * dpm_oracle.c -- FP64 single-threaded reference transport (TEST INFRASTRUCTURE).
 *
 * Test infrastructure only: the product path never links, loads or calls this
 * file.  It is written directly from the model definitions (one closed form
 * per physical process, rejection sampling, exact voxel ray-marching) with no
 * tables, no blocking and no reordering, so that each function can be read
 * against its definition.  See dpm_oracle.h for the model summary.
 *
 * Citations are to the paper (Jia et al., "Development of a GPU-based Monte
 * Carlo dose calculation code for coupled electron-photon transport"):
 *   Sec. 2.1  DPM scheme: condensed history for elastic scattering, detailed
 *             hard inelastic collisions and bremsstrahlung above cut-offs,
 *             CSDA below them, Woodcock tracking for photons;
 *   Sec. 2.2  one source history plus all its secondaries, secondaries kept on
 *             a stack until it is empty;
 *   Sec. 2.4  RANECU generator; dose accumulated per voxel;
 *   Sec. 3    point source, field at SAD 100 cm, absorption energies 200 keV
 *             (electrons) and 50 keV (photons); uncertainty sigma_D per voxel.
 * The paper defines no cross sections; the closed forms used here are the
 * model this project adopts in their place (each named at its function).
 */
#include "dpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
static const double MC2 = 0.51099895;          /* electron rest energy, MeV */
static const double RE = 2.8179403262e-13;     /* classical electron radius, cm */
static const double ALPHA = 1.0 / 137.035999084;
static const double NAV = 6.02214076e23;       /* Avogadro, 1/mol */
static const double PI = 3.14159265358979323846;

/* ======================================================================= */
/* RANECU: combination of two multiplicative congruential generators        */
/* (L'Ecuyer 1988), moduli 2147483563 and 2147483399, multipliers 40014 and */
/* 40692, products reduced without overflow by Schrage's decomposition.     */
/* ======================================================================= */
typedef struct { int32_t s1, s2; } ranecu;

static double ranecu_next(ranecu *r) {
    int32_t k = r->s1 / 53668;
    r->s1 = 40014 * (r->s1 - k * 53668) - k * 12211;
    if (r->s1 < 0) r->s1 += 2147483563;
    k = r->s2 / 52774;
    r->s2 = 40692 * (r->s2 - k * 52774) - k * 3791;
    if (r->s2 < 0) r->s2 += 2147483399;
    int32_t z = r->s1 - r->s2;
    if (z < 1) z += 2147483562;
    return (double)z * 4.656613057391769e-10; /* 1/2147483563 */
}

/* Seeds for history h: SplitMix64 of (seed, h), reduced into each
   generator's range [1, m-1]. */
static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void ranecu_seed(ranecu *r, uint64_t seed, uint64_t h) {
    uint64_t s = seed * 0xD1B54A32D192ED03ULL ^ (h + 0x632BE59BD9B4E019ULL);
    uint64_t a = splitmix64(&s), b = splitmix64(&s);
    r->s1 = (int32_t)(1 + a % 2147483562ULL);
    r->s2 = (int32_t)(1 + b % 2147483398ULL);
}

void or_ranecu_stream(int32_t s1, int32_t s2, int n, double *out, int32_t *state_out) {
    ranecu r = {s1, s2};
    for (int i = 0; i < n; i++) out[i] = ranecu_next(&r);
    if (state_out) { state_out[0] = r.s1; state_out[1] = r.s2; }
}

/* ======================================================================= */
/* Gauss-Legendre quadrature, 16 nodes on [-1, 1]; nodes are the roots of  */
/* P_16 found by Newton's method from the usual cosine starting guesses.    */
/* ======================================================================= */
#define GLN 16
static double gl_x[GLN], gl_w[GLN];
static int gl_ready = 0;

static void gl_init(void) {
    if (gl_ready) return;
    for (int i = 0; i < (GLN + 1) / 2; i++) {
        double z = cos(PI * (i + 0.75) / (GLN + 0.5)), z1, pp;
        do {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= GLN; j++) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = GLN * (z * p1 - p2) / (z * z - 1.0);
            z1 = z;
            z = z1 - p1 / pp;
        } while (fabs(z - z1) > 1e-15);
        gl_x[i] = -z;
        gl_x[GLN - 1 - i] = z;
        gl_w[i] = gl_w[GLN - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    gl_ready = 1;
}

typedef double (*fn1)(double x, const void *ctx);

static double gl_interval(fn1 f, const void *ctx, double a, double b) {
    double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GLN; i++) s += gl_w[i] * f(c + h * gl_x[i], ctx);
    return s * h;
}

/* Composite rule: n equal pieces, and optionally `grade` geometrically
   shrinking pieces toward each end (for integrable end-point singularities). */
static double gl_composite(fn1 f, const void *ctx, double a, double b, int n, int grade) {
    gl_init();
    if (!(b > a)) return 0.0;
    double s = 0.0;
    if (grade > 0) {
        double c = 0.5 * (a + b), w = 0.5 * (b - a);
        for (int k = 0; k < grade; k++) {
            double hi = w * ldexp(1.0, -k), lo = w * ldexp(1.0, -k - 1);
            s += gl_interval(f, ctx, a + lo, a + hi);   /* left end  */
            s += gl_interval(f, ctx, b - hi, b - lo);   /* right end */
        }
        (void)c;
        return s;
    }
    double h = (b - a) / n;
    for (int i = 0; i < n; i++) s += gl_interval(f, ctx, a + i * h, a + (i + 1) * h);
    return s;
}

static double poly_test(double x, const void *ctx) {
    int deg = *(const int *)ctx;
    return pow(x, deg);
}

/* which >= 0: integral of x^which over [a, b] with one 16-point interval. */
double or_gl_integrate_test(int which, double a, double b) {
    gl_init();
    return gl_interval(poly_test, &which, a, b);
}

/* ======================================================================= */
/* Material constants derived from the element list                         */
/* ======================================================================= */
static double mat_z_over_a(const or_material *m) {
    double s = 0;
    for (int i = 0; i < m->n_elem; i++) s += m->w[i] * m->Z[i] / m->A[i];
    return s;
}

/* Radiation length of one element: Dahl's fit, 716.4 A / (Z(Z+1) ln(287/sqrt Z)) g/cm^2. */
double or_x0(const or_material *m) {
    double inv = 0;
    for (int i = 0; i < m->n_elem; i++) {
        double Z = m->Z[i];
        double x0 = 716.4 * m->A[i] / (Z * (Z + 1.0) * log(287.0 / sqrt(Z)));
        inv += m->w[i] / x0;
    }
    return 1.0 / inv;
}

/* ======================================================================= */
/* Photons                                                                  */
/* ======================================================================= */

/* Klein-Nishina total cross section per free electron (cm^2). */
double or_kn_sigma(double E) {
    double k = E / MC2, l = log1p(2.0 * k);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
    return 2.0 * PI * RE * RE * (t1 + t2 - t3);
}

/* Klein-Nishina d(sigma)/d(eps), eps = E'/E in [1/(1+2k), 1]:
   (pi re^2 / k) (eps + 1/eps - sin^2 theta), 1 - cos theta = (1/eps - 1)/k. */
double or_kn_dsde(double E, double eps) {
    double k = E / MC2;
    if (eps < 1.0 / (1.0 + 2.0 * k) || eps > 1.0) return 0.0;
    double omc = (1.0 / eps - 1.0) / k;
    double sin2 = omc * (2.0 - omc);
    return PI * RE * RE / k * (eps + 1.0 / eps - sin2);
}

/* Cumulative fraction of the Klein-Nishina eps distribution below eps, from
   the antiderivative of eps + (c^2-1) + (1-2c/k)/eps + 1/(k eps)^2 with
   c = 1 + 1/k (the integrand above written in powers of eps). */
static double kn_antider(double k, double e) {
    double c = 1.0 + 1.0 / k;
    return 0.5 * e * e + (c * c - 1.0) * e + (1.0 - 2.0 * c / k) * log(e) - 1.0 / (k * k * e);
}
double or_kn_cdf(double E, double eps) {
    double k = E / MC2, e0 = 1.0 / (1.0 + 2.0 * k);
    if (eps <= e0) return 0.0;
    if (eps >= 1.0) return 1.0;
    return (kn_antider(k, eps) - kn_antider(k, e0)) / (kn_antider(k, 1.0) - kn_antider(k, e0));
}

/* Compton mass attenuation: N_A (Z/A) sigma_KN (cm^2/g). */
double or_mu_compton(const or_material *m, double E) {
    return NAV * mat_z_over_a(m) * or_kn_sigma(E);
}

/* Photoelectric mass attenuation: c_pe * sum_i w_i Z_i^4 / A_i / E^3. */
double or_mu_photo(const or_material *m, double E, double c_pe) {
    double s = 0;
    for (int i = 0; i < m->n_elem; i++) s += m->w[i] * pow(m->Z[i], 4) / m->A[i];
    return c_pe * s / (E * E * E);
}

/* Bethe-Heitler (unscreened, extreme-relativistic) pair spectrum shape in the
   electron's share eps of the photon energy, without the 4 Z(Z+1) alpha re^2
   prefactor: [eps^2 + (1-eps)^2 + (2/3) eps (1-eps)] (ln(2 k eps (1-eps)) - 1/2),
   clamped at zero when `clamp` is set. */
double or_pair_dsde_shape(double kappa, double eps, int clamp) {
    double pe = eps * eps + (1 - eps) * (1 - eps) + (2.0 / 3.0) * eps * (1 - eps);
    double lg = log(2.0 * kappa * eps * (1 - eps)) - 0.5;
    if (clamp && lg < 0) lg = 0;
    return pe * lg;
}

typedef struct { double kappa; int clamp; } pair_ctx;
static double pair_f(double e, const void *c) {
    const pair_ctx *p = (const pair_ctx *)c;
    return or_pair_dsde_shape(p->kappa, e, p->clamp);
}

/* 4 * integral of the shape over [lo, hi].  With clamp = 0 and [0, 1] this is
   28/9 ln(2k) - 218/27; the physical cross section integrates the clamped
   shape over the kinematic range eps in [1/k, 1-1/k]. */
double or_pair_integral(double kappa, double lo, double hi, int clamp) {
    pair_ctx c = {kappa, clamp};
    if (!clamp) return 4.0 * gl_composite(pair_f, &c, lo, hi, 0, 40);
    /* the clamped shape is positive where eps(1-eps) > e^{1/2}/(2k) */
    double disc = 1.0 - 2.0 * exp(0.5) / kappa;
    if (disc <= 0) return 0.0;
    double em = 0.5 * (1 - sqrt(disc)), ep = 0.5 * (1 + sqrt(disc));
    double a = lo > em ? lo : em, b = hi < ep ? hi : ep;
    if (!(b > a)) return 0.0;
    return 4.0 * gl_composite(pair_f, &c, a, b, 8, 0);
}

/* Pair mass attenuation: N_A sum_i w_i Z_i(Z_i+1)/A_i alpha re^2 * I(k). */
double or_mu_pair(const or_material *m, double E) {
    double k = E / MC2;
    if (k <= 2.0) return 0.0;
    double zz = 0;
    for (int i = 0; i < m->n_elem; i++) zz += m->w[i] * m->Z[i] * (m->Z[i] + 1) / m->A[i];
    return NAV * zz * ALPHA * RE * RE * or_pair_integral(k, 1.0 / k, 1.0 - 1.0 / k, 1);
}

/* ======================================================================= */
/* Electrons                                                                */
/* ======================================================================= */

/* Plasma energy hbar*omega_p = hbar c sqrt(4 pi n_e r_e) of the material at
   its density-effect density, in eV (n_e electrons per cm^3). */
double or_plasma_energy_ev(const or_material *m) {
    const double HBARC = 1.973269804e-11; /* MeV cm */
    double ne = m->rho_de * NAV * mat_z_over_a(m);
    return HBARC * sqrt(4.0 * PI * ne * RE) * 1e6;
}

/* Density-effect correction delta of the collision stopping power, by the
   general formula of Sternheimer and Peierls (1971) for condensed media,
   in X = log10(beta gamma) = log10(p/mc):
     Cbar = 2 ln(I / hbar omega_p) + 1;
     I < 100 eV:  X1 = 2, X0 = 0.2 if Cbar < 3.681 else 0.326 Cbar - 1.0;
     I >= 100 eV: X1 = 3, X0 = 0.2 if Cbar < 5.215 else 0.326 Cbar - 1.5;
     delta = 0 below X0; 2 ln10 X - Cbar + a (X1 - X)^3 on [X0, X1) with a
     making delta vanish at X0; 2 ln10 X - Cbar from X1 on.
   Zero when the material has no density-effect density. */
double or_density_delta(const or_material *m, double T) {
    if (!(m->rho_de > 0.0)) return 0.0;
    double cbar = 2.0 * log(m->i_ev / or_plasma_energy_ev(m)) + 1.0;
    double x0, x1;
    if (m->i_ev < 100.0) {
        x1 = 2.0;
        x0 = cbar < 3.681 ? 0.2 : 0.326 * cbar - 1.0;
    } else {
        x1 = 3.0;
        x0 = cbar < 5.215 ? 0.2 : 0.326 * cbar - 1.5;
    }
    double two_ln10 = 2.0 * log(10.0);
    double t = T / MC2;
    double X = 0.5 * log10(t * (t + 2.0)); /* (beta gamma)^2 = t (t + 2) */
    if (X < x0) return 0.0;
    double lin = two_ln10 * X - cbar;
    if (X >= x1) return lin;
    double a = (cbar - two_ln10 * x0) / ((x1 - x0) * (x1 - x0) * (x1 - x0));
    return lin + a * (x1 - X) * (x1 - X) * (x1 - X);
}

/* Restricted collision stopping power (Bethe, electrons), MeV cm^2/g, for
   energy transfers below d = min(wcc, T/2):
   2 pi re^2 mc^2 N_A (Z/A)/beta^2 [ ln(2(t+2)/(I/mc^2)^2) - 1 - beta^2
       + ln((t-d)d) + t/(t-d) + (d^2/2 + (2t+1) ln(1-d/t))/gamma^2 - delta ],
   t = T/mc^2, d in units of mc^2, delta the density effect (zero unless the
   material asks for it).  With d = t/2 this is the unrestricted form. */
double or_scol(const or_material *m, double T, double wcc) {
    double t = T / MC2, g = t + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double I = m->i_ev * 1e-6 / MC2;
    double d = wcc / MC2;
    if (d > 0.5 * t) d = 0.5 * t;
    double br = log(2.0 * (t + 2.0) / (I * I)) - 1.0 - b2 + log((t - d) * d) + t / (t - d)
                + (0.5 * d * d + (2.0 * t + 1.0) * log(1.0 - d / t)) / (g * g) - or_density_delta(m, T);
    return 2.0 * PI * RE * RE * MC2 * NAV * mat_z_over_a(m) / b2 * br;
}

/* Restricted radiative stopping power from the simplified spectrum
   dsigma/dk = (1/(X0 k)) (4/3 - 4/3 y + y^2), y = k/(T+mc^2), integrated k dsigma
   over k < min(wcr, T):  (E/X0) [4/3 yc - 2/3 yc^2 + yc^3/3]. */
double or_srad(const or_material *m, double T, double wcr) {
    double E = T + MC2, kc = wcr < T ? wcr : T, y = kc / E;
    return E / or_x0(m) * ((4.0 / 3.0) * y - (2.0 / 3.0) * y * y + y * y * y / 3.0);
}

/* Moller d(sigma)/dW per gram (cm^2/g/MeV), W the energy given to the
   secondary electron, eps = W/T:
   N_A (Z/A) 2 pi re^2 mc^2/(beta^2 T^2) [1/eps^2 + 1/(1-eps)^2 + (t/g)^2 - (2t+1)/g^2/(eps(1-eps))]. */
double or_moller_dsdw(const or_material *m, double T, double W) {
    double t = T / MC2, g = t + 1.0, b2 = 1.0 - 1.0 / (g * g), e = W / T;
    double br = 1.0 / (e * e) + 1.0 / ((1 - e) * (1 - e)) + (t / g) * (t / g) - (2 * t + 1) / (g * g) / (e * (1 - e));
    return NAV * mat_z_over_a(m) * 2.0 * PI * RE * RE * MC2 / (b2 * T * T) * br;
}

/* Hard Moller cross section per gram: the integral of the above over
   W in [wcc, T/2], in closed form. */
double or_moller_sigma(const or_material *m, double T, double wcc) {
    if (T <= 2.0 * wcc) return 0.0;
    double t = T / MC2, g = t + 1.0, b2 = 1.0 - 1.0 / (g * g), ec = wcc / T;
    double br = (1.0 / ec - 2.0) + (2.0 - 1.0 / (1.0 - ec)) + (t / g) * (t / g) * (0.5 - ec)
                - (2 * t + 1) / (g * g) * log((1.0 - ec) / ec);
    return NAV * mat_z_over_a(m) * 2.0 * PI * RE * RE * MC2 / (b2 * T) * br;
}

/* Simplified bremsstrahlung spectrum per gram (cm^2/g/MeV). */
double or_brems_dsdk(const or_material *m, double T, double k) {
    double y = k / (T + MC2);
    return (4.0 / 3.0 - (4.0 / 3.0) * y + y * y) / (or_x0(m) * k);
}

/* Hard bremsstrahlung cross section per gram, k in [wcr, T], closed form. */
double or_brems_sigma(const or_material *m, double T, double wcr) {
    if (T <= wcr) return 0.0;
    double E = T + MC2;
    return ((4.0 / 3.0) * log(T / wcr) - (4.0 / 3.0) * (T - wcr) / E + (T * T - wcr * wcr) / (2.0 * E * E)) / or_x0(m);
}

/* Inverse transport mean free path per gram (cm^2/g) for screened Rutherford
   scattering Z(Z+1) re^2/(beta^4 gamma^2) / (1 - mu + 2 eta)^2 with Moliere's
   screening eta = 1/4 (alpha Z^{1/3}/(0.885 beta gamma))^2 (1.13 + 3.76 (alpha Z/beta)^2):
   sum_i N_A w_i/A_i 2 pi Z(Z+1) re^2/(beta^4 gamma^2) [ln(1+1/eta) - 1/(1+eta)]. */
double or_lambda1_inv(const or_material *m, double T) {
    double t = T / MC2, g = t + 1.0, b2 = 1.0 - 1.0 / (g * g), bg2 = t * (t + 2.0);
    double s = 0;
    for (int i = 0; i < m->n_elem; i++) {
        double Z = m->Z[i];
        double chi = ALPHA * cbrt(Z) / 0.885;
        double eta = 0.25 * chi * chi / bg2 * (1.13 + 3.76 * ALPHA * ALPHA * Z * Z / b2);
        double br = log1p(1.0 / eta) - 1.0 / (1.0 + eta);
        s += NAV * m->w[i] / m->A[i] * 2.0 * PI * Z * (Z + 1.0) * RE * RE / (b2 * bg2) * br;
    }
    return s;
}

typedef struct { const or_material *m; const or_params *p; } sp_ctx;

/* integrand of the range in u = ln T: T / S(T) */
static double range_f(double u, const void *c) {
    const sp_ctx *s = (const sp_ctx *)c;
    double T = exp(u);
    return T / (or_scol(s->m, T, s->p->wcc) + or_srad(s->m, T, s->p->wcr));
}

/* CSDA mass path (g/cm^2) to slow down from T_hi to T_lo: integral of dT/S(T)
   with S the restricted collision + restricted radiative stopping power. */
static double range_piece(const sp_ctx *c, double T_lo, double T_hi) {
    double a = log(T_lo), b = log(T_hi);
    int n = (int)ceil((b - a) / 0.05);
    if (n < 1) n = 1;
    return gl_composite(range_f, c, a, b, n, 0);
}

/* The stopping power has kinks where the cuts switch regime (T = 2 wcc for
   collisions, T = wcr for radiation), so the integral is split there. */
double or_csda_path(const or_material *m, const or_params *p, double T_lo, double T_hi) {
    if (!(T_hi > T_lo)) return 0.0;
    sp_ctx c = {m, p};
    double cuts[2] = {p->wcr < 2.0 * p->wcc ? p->wcr : 2.0 * p->wcc, p->wcr < 2.0 * p->wcc ? 2.0 * p->wcc : p->wcr};
    double s = 0.0, lo = T_lo;
    for (int i = 0; i < 2; i++) {
        if (cuts[i] > lo && cuts[i] < T_hi) {
            s += range_piece(&c, lo, cuts[i]);
            lo = cuts[i];
        }
    }
    return s + range_piece(&c, lo, T_hi);
}

/* Kinetic energy after a CSDA mass path: the T' with or_csda_path(T', T) =
   mass_path, by Newton's method (derivative -1/S(T')). */
double or_csda_energy(const or_material *m, const or_params *p, double T, double mass_path) {
    if (mass_path <= 0) return T;
    double S = or_scol(m, T, p->wcc) + or_srad(m, T, p->wcr);
    double Tp = T - mass_path * S;
    if (Tp < 0.5 * T) Tp = 0.5 * T;
    for (int it = 0; it < 60; it++) {
        double g = or_csda_path(m, p, Tp, T) - mass_path;
        double Sp = or_scol(m, Tp, p->wcc) + or_srad(m, Tp, p->wcr);
        double step = g * Sp;
        double Tn = Tp + step;
        if (Tn <= 0.25 * Tp) Tn = 0.25 * Tp;
        if (Tn > T) Tn = T;
        if (fabs(Tn - Tp) <= 1e-14 * T) { Tp = Tn; break; }
        Tp = Tn;
    }
    return Tp;
}

/* Random-hinge angular distribution: p(x) = 2A(1+A)/(x+2A)^2 on x = 1-mu in
   [0, 2], whose mean is 2A[(1+A) ln(1+1/A) - 1].  For A >= 100 the bracket
   cancels badly, so the mean and its derivative use the expansion in 1/A,
   1 - sum_{n>=3} 2(-1)^(n+1) A^{-(n-2)}/(n(n-1)). */
static void msc_mean_and_slope(double A, double *mean, double *slope) {
    if (A < 100.0) {
        double l = log1p(1.0 / A);
        *mean = 2.0 * A * ((1.0 + A) * l - 1.0);
        *slope = 2.0 * (1.0 + 2.0 * A) * l - 4.0;
        return;
    }
    double x = 1.0 / A, m = 1.0, d = 0.0, xp = 1.0;
    for (int n = 3; n <= 14; n++) {
        double c = ((n & 1) ? -2.0 : 2.0) / (n * (n - 1.0));  /* coefficient of x^(n-2) */
        d += c * (n - 2) * xp * x * x;                        /* d/dA of c x^(n-2) is -(n-2) c x^(n-1) ... */
        xp *= x;
        m += c * xp;
    }
    *mean = m;
    *slope = -d;
}

double or_msc_mean(double A) {
    double m, s;
    msc_mean_and_slope(A, &m, &s);
    return m;
}

/* A such that or_msc_mean(A) = q (0 < q < 1): safeguarded Newton in ln A. */
double or_msc_A(double q) {
    if (q <= 0) return 0.0;
    if (q >= 1.0 - 1e-12) return 1.0 / (3.0 * (1.0 - q) + 1e-300);
    double lo = -90.0, hi = 40.0, x = log(q);
    for (int it = 0; it < 300; it++) {
        double A = exp(x), m, s;
        msc_mean_and_slope(A, &m, &s);
        double h = m - q;
        if (h > 0) hi = x; else lo = x;
        double dh = A * s;
        double xn = (dh > 0) ? x - h / dh : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) < 1e-14 * (1.0 + fabs(x)) || hi - lo < 1e-14) { x = xn; break; }
        x = xn;
    }
    return exp(x);
}

/* Synthetic 6 MV spectrum f(E) ~ (1 - E/6) E^{-1/2} on [0.25, 6] MeV: with
   t = sqrt(E) the cumulative integral is 2t - t^3/9. */
static double spec_F(double t) { return 2.0 * t - t * t * t / 9.0; }
double or_spectrum_cdf(double E) {
    if (E <= 0.25) return 0.0;
    if (E >= 6.0) return 1.0;
    double t0 = 0.5, t1 = sqrt(6.0);
    return (spec_F(sqrt(E)) - spec_F(t0)) / (spec_F(t1) - spec_F(t0));
}

/* ======================================================================= */
/* Samplers (rejection methods written from each density)                   */
/* ======================================================================= */

/* Klein-Nishina eps: propose from 1/eps + eps (a two-part mixture with
   inverse transforms), accept with the remaining factor
   1 - eps sin^2(theta)/(1 + eps^2)  (Butcher & Messel's decomposition). */
static double sample_kn(double E, ranecu *r) {
    double k = E / MC2, e0 = 1.0 / (1.0 + 2.0 * k);
    double a1 = -log(e0), a2 = 0.5 * (1.0 - e0 * e0);
    for (;;) {
        double x1 = ranecu_next(r), x2 = ranecu_next(r), x3 = ranecu_next(r);
        double e;
        if (x1 * (a1 + a2) < a1) e = exp(-a1 * x2);
        else e = sqrt(e0 * e0 + (1.0 - e0 * e0) * x2);
        double omc = (1.0 - e) / (k * e);
        double sin2 = omc * (2.0 - omc);
        if (x3 <= 1.0 - e * sin2 / (1.0 + e * e)) return e;
    }
}

/* Moller eps = W/T in [wcc/T, 1/2]: propose from 1/eps^2, accept with
   eps^2 [bracket] / (9/4), the bracket of or_moller_dsdw. */
static double sample_moller(double T, double wcc, ranecu *r) {
    double t = T / MC2, g = t + 1.0, ec = wcc / T;
    for (;;) {
        double x1 = ranecu_next(r), x2 = ranecu_next(r);
        double e = 1.0 / (1.0 / ec - x1 * (1.0 / ec - 2.0));
        double q = e / (1.0 - e);
        double f = 1.0 + q * q + (t / g) * (t / g) * e * e - (2 * t + 1) / (g * g) * q;
        if (x2 * 2.25 <= f) return e;
    }
}

/* Bremsstrahlung k in [wcr, T]: propose from 1/k, accept with
   (4/3 - 4/3 y + y^2)/(4/3). */
static double sample_brems(double T, double wcr, ranecu *r) {
    double E = T + MC2;
    for (;;) {
        double x1 = ranecu_next(r), x2 = ranecu_next(r);
        double k = wcr * exp(x1 * log(T / wcr));
        double y = k / E;
        if (x2 * (4.0 / 3.0) <= 4.0 / 3.0 - (4.0 / 3.0) * y + y * y) return k;
    }
}

/* Pair eps (electron share): uniform over the region where the clamped
   shape is positive within [1/k, 1-1/k], accept with shape / (ln(k/2) - 1/2)
   (the polynomial factor is at most 1 and the log factor peaks at eps = 1/2). */
static double sample_pair(double E, ranecu *r) {
    double k = E / MC2;
    double disc = 1.0 - 2.0 * exp(0.5) / k;
    double em = 0.5 * (1 - sqrt(disc)), ep = 0.5 * (1 + sqrt(disc));
    double a = 1.0 / k > em ? 1.0 / k : em, b = 1.0 - 1.0 / k < ep ? 1.0 - 1.0 / k : ep;
    double fmax = log(0.5 * k) - 0.5;
    for (;;) {
        double x1 = ranecu_next(r), x2 = ranecu_next(r);
        double e = a + (b - a) * x1;
        if (x2 * fmax <= or_pair_dsde_shape(k, e, 1)) return e;
    }
}

/* 1 - mu from the hinge distribution by its inverse CDF. */
static double sample_msc(double A, ranecu *r) {
    double x = ranecu_next(r);
    return 2.0 * A * x / (1.0 + A - x);
}

/* Photoelectron direction (the DPM physics of Sec. 2.1 gives the K-shell
   photoelectron Sauter's angular distribution; optional here, OR_SAUTER):
   dsigma/dOmega ~ sin^2(th)/(1 - b cos th)^4 [1 + g(g-1)(g-2)(1 - b cos th)/2]
   with b, g the electron's speed and Lorentz factor.  In nu = 1 - cos th,
   with A = 1/b - 1 and B = b g(g-1)(g-2)/2, the density is
   p(nu) ~ nu(2 - nu) [1/(A+nu)^4 + B/(A+nu)^3] on [0, 2].  Propose
   q(nu) ~ nu/(A+nu)^3, whose CDF is (x/x_max)^2 in x = nu/(A+nu)
   (x_max = 2/(A+2)), and accept with (2 - nu)((1-x)/A + B) over its bound
   2(1/A + max(B, 0)).  Returns nu. */
static double sample_sauter(double T, ranecu *r) {
    double g = 1.0 + T / MC2, b = sqrt(T * (T + 2.0 * MC2)) / (T + MC2);
    double A = 1.0 / b - 1.0, B = 0.5 * b * g * (g - 1.0) * (g - 2.0);
    double xm = 2.0 / (A + 2.0), M = 2.0 * (1.0 / A + (B > 0 ? B : 0.0));
    for (;;) {
        double x = xm * sqrt(ranecu_next(r));
        double nu = A * x / (1.0 - x);
        if (ranecu_next(r) * M <= (2.0 - nu) * ((1.0 - x) / A + B)) return nu;
    }
}

/* 6 MV energy by bisection on the CDF. */
static double sample_spectrum(ranecu *r) {
    double u = ranecu_next(r);
    double t0 = 0.5, t1 = sqrt(6.0);
    double target = spec_F(t0) + u * (spec_F(t1) - spec_F(t0));
    double lo = t0, hi = t1;
    for (int i = 0; i < 80; i++) {
        double mid = 0.5 * (lo + hi);
        if (spec_F(mid) < target) lo = mid; else hi = mid;
    }
    double t = 0.5 * (lo + hi);
    return t * t;
}

static void isotropic_direction(ranecu *r, double d[3]);

void or_sample(int which, double a, double b, const or_material *m, uint64_t n, uint64_t seed, double *out) {
    (void)m;
    ranecu r;
    ranecu_seed(&r, seed, 0x5A5A5A5AULL + (uint64_t)which);
    for (uint64_t i = 0; i < n; i++) {
        switch (which) {
            case OR_S_KN: out[i] = sample_kn(a, &r); break;
            case OR_S_MOLLER: out[i] = sample_moller(a, b, &r); break;
            case OR_S_BREMS: out[i] = sample_brems(a, b, &r); break;
            case OR_S_PAIR: out[i] = sample_pair(a, &r); break;
            case OR_S_MSC: out[i] = sample_msc(a, &r); break;
            case OR_S_SPECTRUM: out[i] = sample_spectrum(&r); break;
            case OR_S_SAUTER: out[i] = sample_sauter(a, &r); break;
            case OR_S_ISO_X:
            case OR_S_ISO_Z: {
                double d[3];
                isotropic_direction(&r, d);
                out[i] = which == OR_S_ISO_X ? d[0] : d[2];
                break;
            }
            default: out[i] = 0;
        }
    }
}

/* ======================================================================= */
/* Geometry                                                                 */
/* ======================================================================= */
typedef struct {
    double x[3], d[3], E;
    int iv[3];
    int type; /* 0 photon, 1 electron, 2 positron */
} part;

static const double INF = 1e300;

static double dist_boundary(const part *p, const or_phantom *ph, int *axis) {
    const double D[3] = {ph->dx, ph->dy, ph->dz};
    double best = INF;
    *axis = -1;
    for (int a = 0; a < 3; a++) {
        double t;
        if (p->d[a] > 0) t = ((p->iv[a] + 1) * D[a] - p->x[a]) / p->d[a];
        else if (p->d[a] < 0) t = (p->iv[a] * D[a] - p->x[a]) / p->d[a];
        else continue;
        if (t < 0) t = 0;
        if (t < best) { best = t; *axis = a; }
    }
    return best;
}

static void move(part *p, double s) {
    for (int a = 0; a < 3; a++) p->x[a] += s * p->d[a];
}

/* Step into the neighbouring voxel across `axis`; 0 if that leaves the phantom. */
static int cross(part *p, const or_phantom *ph, int axis) {
    const double D[3] = {ph->dx, ph->dy, ph->dz};
    const int N[3] = {ph->nx, ph->ny, ph->nz};
    if (p->d[axis] > 0) { p->iv[axis] += 1; p->x[axis] = p->iv[axis] * D[axis]; }
    else { p->x[axis] = p->iv[axis] * D[axis]; p->iv[axis] -= 1; }
    return p->iv[axis] >= 0 && p->iv[axis] < N[axis];
}

static long lin(const part *p, const or_phantom *ph) {
    return p->iv[0] + (long)ph->nx * (p->iv[1] + (long)ph->ny * p->iv[2]);
}

/* Rotate direction d by polar cosine c and azimuth phi. */
static void rotate(double d[3], double c, double phi) {
    if (c > 1) c = 1;
    if (c < -1) c = -1;
    double s = sqrt(1.0 - c * c), cp = cos(phi), sp = sin(phi);
    double u = d[0], v = d[1], w = d[2];
    double r = sqrt(u * u + v * v);
    if (r < 1e-10) {
        d[0] = s * cp;
        d[1] = s * sp;
        d[2] = (w >= 0 ? 1.0 : -1.0) * c;
    } else {
        d[0] = u * c + s * (u * w * cp - v * sp) / r;
        d[1] = v * c + s * (v * w * cp + u * sp) / r;
        d[2] = w * c - s * r * cp;
    }
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= n; d[1] /= n; d[2] /= n;
}

/* Compton scattering of a photon of energy E into eps E (Sec. 2.1,
   Klein-Nishina): the photon turns by cos theta = 1 - (1/eps - 1)/kappa at
   azimuth phi; the electron takes T = E - eps E at the polar angle fixed by
   momentum conservation, cos theta_e = (E - eps E cos theta)/p_e, on the
   opposite azimuth.  d_g and d_e start as the photon's direction. */
static void compton_kinematics(double E, double e, double phi, double d_g[3], double d_e[3], double *Ep,
                               double *T) {
    *Ep = e * E;
    *T = E - *Ep;
    double cth = 1.0 - (1.0 / e - 1.0) / (E / MC2);
    double pe = sqrt(*T * (*T + 2.0 * MC2));
    double ce = (E - *Ep * cth) / pe;
    rotate(d_e, ce, phi + PI);
    rotate(d_g, cth, phi);
}

/* Moller collision of an electron of kinetic energy T giving W to the
   secondary (Sec. 2.1): both polar angles from the two-body kinematics of a
   collision with an electron at rest, cos^2 theta = W (T + 2 mc^2) /
   (T (W + 2 mc^2)) for the secondary and the same with T - W for the
   primary, on opposite azimuths.  d_p and d_s start as the primary's
   direction. */
static void moller_kinematics(double T, double W, double phi, double d_p[3], double d_s[3]) {
    double Tp = T - W;
    double cs = sqrt(W * (T + 2.0 * MC2) / (T * (W + 2.0 * MC2)));
    double cp = sqrt(Tp * (T + 2.0 * MC2) / (T * (Tp + 2.0 * MC2)));
    rotate(d_s, cs, phi);
    rotate(d_p, cp, phi + PI);
}

/* Test hook: one interaction's outgoing particles from an incoming
   direction d_in, for the conservation-law pins.  which 0: Compton (a = E,
   b = eps); 1: Moller (a = T, b = W).  out = {E1, d1[3], E2, d2[3]}: the
   scattered photon then the electron, or the primary then the secondary. */
void or_kinematics(int which, double a, double b, double phi, const double d_in[3], double out[8]) {
    double d1[3] = {d_in[0], d_in[1], d_in[2]}, d2[3] = {d_in[0], d_in[1], d_in[2]};
    if (which == 0) {
        double Ep, T;
        compton_kinematics(a, b, phi, d1, d2, &Ep, &T);
        out[0] = Ep;
        out[4] = T;
    } else {
        moller_kinematics(a, b, phi, d1, d2);
        out[0] = a - b;
        out[4] = b;
    }
    for (int k = 0; k < 3; k++) {
        out[1 + k] = d1[k];
        out[5 + k] = d2[k];
    }
}

/* ======================================================================= */
/* Transport                                                                */
/* ======================================================================= */
#define STACK_MAX 4096
#define OR_MAXMAT 16

typedef struct {
    const or_phantom *ph;
    const or_material *mats;
    int n_mat;
    const or_params *p;
    ranecu rng;
    /* per-history tally */
    double *hE;
    long *touched;
    long n_touched, cap_touched;
    double h_dep, h_esc;
    long last_v;
    part stack[STACK_MAX];
    int sp;
    int err;
    or_stats *st;
} tctx;

static void deposit(tctx *c, long v, double e) {
    if (e == 0) return;
    if (c->hE[v] == 0.0) {
        if (c->n_touched == c->cap_touched) {
            c->cap_touched *= 2;
            c->touched = (long *)realloc(c->touched, sizeof(long) * c->cap_touched);
        }
        c->touched[c->n_touched++] = v;
    }
    c->hE[v] += e;
    c->h_dep += e;
    c->st->n_dep++;
    if (v != c->last_v) { c->st->n_dep_runs++; c->last_v = v; }
}

static void push(tctx *c, const part *q) {
    if (c->sp >= STACK_MAX) { c->err = 1; return; }
    c->stack[c->sp++] = *q;
    if (q->type == 0) c->st->n_sec_g++; else c->st->n_sec_e++;
    if (q->type == 2) c->st->n_positrons++;
}

static void escape(tctx *c, double e) { c->h_esc += e; }

/* Isotropic direction: cos theta uniform on [-1, 1], azimuth uniform. */
static void isotropic_direction(ranecu *r, double d[3]) {
    double cz = 2.0 * ranecu_next(r) - 1.0, phi = 2.0 * PI * ranecu_next(r);
    double sz = sqrt(1.0 - cz * cz);
    d[0] = sz * cos(phi); d[1] = sz * sin(phi); d[2] = cz;
}

/* Two annihilation photons, isotropic and back to back, at the positron's
   final position. */
static void annihilate(tctx *c, const part *p) {
    part g = *p;
    g.type = 0;
    g.E = MC2;
    isotropic_direction(&c->rng, g.d);
    push(c, &g);
    g.d[0] = -g.d[0]; g.d[1] = -g.d[1]; g.d[2] = -g.d[2];
    push(c, &g);
}

/* A newly created charged particle: transported if above the absorption
   energy, otherwise deposited on the spot (positrons then annihilate). */
static void emit_charged(tctx *c, part *q) {
    if (q->E > c->p->eabs_e) { push(c, q); return; }
    deposit(c, lin(q, c->ph), q->E);
    if (q->type == 2) annihilate(c, q);
}

static void emit_photon(tctx *c, part *q) {
    if (c->p->flags & OR_NO_SECONDARY_PHOTONS) { escape(c, q->E); return; }
    if (q->E > c->p->eabs_g) { push(c, q); return; }
    deposit(c, lin(q, c->ph), q->E);
}

/* Photon history segment: exact ray-march through voxels with the real
   attenuation coefficient of each voxel (Sec. 2.1 uses Woodcock tracking;
   the oracle does the exact march so that the GPU's majorant logic is
   checked against an independent method).  Returns 1 if the first flight
   left the phantom without interacting (used by or_uncollided). */
static int transport_photon(tctx *c, part *p, int first_flight_only) {
    const or_phantom *ph = c->ph;
    double muc[OR_MAXMAT], mup[OR_MAXMAT], mur[OR_MAXMAT], mut[OR_MAXMAT];
    for (;;) {
        if (p->E <= c->p->eabs_g) { deposit(c, lin(p, ph), p->E); return 0; }
        for (int m = 0; m < c->n_mat; m++) {
            muc[m] = or_mu_compton(&c->mats[m], p->E);
            mup[m] = or_mu_photo(&c->mats[m], p->E, c->p->c_pe);
            mur[m] = or_mu_pair(&c->mats[m], p->E);
            mut[m] = muc[m] + mup[m] + mur[m];
        }
        double tau = -log(ranecu_next(&c->rng));
        int m;
        for (;;) {
            long v = lin(p, ph);
            m = ph->mat[v];
            double mu = (double)ph->rho[v] * mut[m];
            int axis;
            double t = dist_boundary(p, ph, &axis);
            c->st->n_g_voxel_steps++;
            if (tau <= mu * t) { move(p, tau / mu); break; }
            tau -= mu * t;
            move(p, t);
            if (!cross(p, ph, axis)) { escape(c, p->E); return 1; }
        }
        if (first_flight_only) return 0;
        c->st->n_g_interactions++;
        long v = lin(p, ph);
        double r = ranecu_next(&c->rng) * mut[m];
        if (r < muc[m]) {
            /* Compton: photon keeps eps E, electron gets the rest */
            double E = p->E, e = sample_kn(E, &c->rng), Ep, T;
            double phi = 2.0 * PI * ranecu_next(&c->rng);
            part el = *p;
            el.type = 1;
            compton_kinematics(E, e, phi, p->d, el.d, &Ep, &T);
            el.E = T;
            emit_charged(c, &el);
            p->E = Ep;
            continue;
        } else if (r < muc[m] + mup[m]) {
            /* photoelectric: the electron takes all the energy, along the
               photon direction or (OR_SAUTER) at Sauter's polar angle */
            part el = *p;
            el.type = 1;
            if ((c->p->flags & OR_SAUTER) && el.E > c->p->eabs_e) {
                double nu = sample_sauter(el.E, &c->rng);
                rotate(el.d, 1.0 - nu, 2.0 * PI * ranecu_next(&c->rng));
            }
            emit_charged(c, &el);
            return 0;
        } else {
            /* pair: electron eps E - mc^2, positron (1-eps) E - mc^2, both
               along the photon direction */
            double E = p->E, e = sample_pair(E, &c->rng);
            part a = *p, b = *p;
            a.type = 1; a.E = e * E - MC2;
            b.type = 2; b.E = (1.0 - e) * E - MC2;
            emit_charged(c, &a);
            emit_charged(c, &b);
            (void)v;
            return 0;
        }
    }
}

static void absorb_charged(tctx *c, part *p) {
    deposit(c, lin(p, c->ph), p->E);
    if (p->type == 2) annihilate(c, p);
}

/* Condensed-history electron (or positron) transport, Sec. 2.1.
   Each step: CSDA step length for a fractional loss f_e (not below eabs_e);
   a hard-event distance from the hard cross section at the step's starting
   energy (a majorant, since that cross section grows with energy); a random
   hinge at a uniform fraction of the step where the multiple-scattering
   deflection is applied; steps stop at voxel boundaries without a deflection
   if the boundary comes before the hinge; at a candidate hard event the
   event is real with probability sigma(T_event)/sigma(T_start) and is then
   Moller or bremsstrahlung in proportion to their cross sections. */
static void transport_electron(tctx *c, part *p) {
    const or_phantom *ph = c->ph;
    const or_params *pr = c->p;
    for (;;) {
        if (p->E <= pr->eabs_e) { absorb_charged(c, p); return; }
        long v = lin(p, ph);
        const or_material *m = &c->mats[ph->mat[v]];
        double rho = ph->rho[v];
        double T = p->E;
        double Tend = (1.0 - pr->f_e) * T;
        if (Tend < pr->eabs_e) Tend = pr->eabs_e;
        double sE = or_csda_path(m, pr, Tend, T) / rho;
        double sig = 0;
        if (!(pr->flags & OR_NO_HARD)) sig = or_moller_sigma(m, T, pr->wcc) + or_brems_sigma(m, T, pr->wcr);
        double xh = ranecu_next(&c->rng);
        double sh = sig > 0 ? -log(xh) / (rho * sig) : INF;
        int hard = sh < sE;
        double s = hard ? sh : sE;
        double tau = ranecu_next(&c->rng);
        int axis, crossed = 0;
        double path;
        double t1 = dist_boundary(p, ph, &axis);
        c->st->n_e_steps++;
        if (t1 <= tau * s) {
            move(p, t1);
            path = t1;
            crossed = 1;
        } else {
            move(p, tau * s);
            path = tau * s;
            if (!(pr->flags & OR_NO_MSC)) {
                double q = -expm1(-rho * s * or_lambda1_inv(m, T));
                double A = or_msc_A(q);
                double x = sample_msc(A, &c->rng);
                double phi = 2.0 * PI * ranecu_next(&c->rng);
                rotate(p->d, 1.0 - x, phi);
            }
            double rest = (1.0 - tau) * s;
            double t2 = dist_boundary(p, ph, &axis);
            if (t2 <= rest) {
                move(p, t2);
                path += t2;
                crossed = 1;
            } else {
                move(p, rest);
                path = s;
            }
        }
        double Tn = (!crossed && !hard) ? Tend : or_csda_energy(m, pr, T, rho * path);
        deposit(c, v, T - Tn);
        c->st->e_path += path;
        p->E = Tn;
        if (crossed) {
            if (!cross(p, ph, axis)) {
                escape(c, p->E + (p->type == 2 ? 2.0 * MC2 : 0.0));
                return;
            }
            continue;
        }
        if (!hard || Tn <= pr->eabs_e) continue;
        /* candidate hard event at energy Tn */
        double sm = or_moller_sigma(m, Tn, pr->wcc), sb = or_brems_sigma(m, Tn, pr->wcr);
        if (ranecu_next(&c->rng) * sig >= sm + sb) continue; /* null event */
        if (ranecu_next(&c->rng) * (sm + sb) < sm) {
            /* Moller: secondary gets W = eps T, primary keeps T - W */
            double e = sample_moller(Tn, pr->wcc, &c->rng), W = e * Tn, Tp = Tn - W;
            double phi = 2.0 * PI * ranecu_next(&c->rng);
            part d = *p;
            d.type = 1;
            d.E = W;
            moller_kinematics(Tn, W, phi, p->d, d.d);
            emit_charged(c, &d);
            p->E = Tp;
        } else {
            /* bremsstrahlung photon along the electron direction */
            double k = sample_brems(Tn, pr->wcr, &c->rng);
            part g = *p;
            g.type = 0;
            g.E = k;
            emit_photon(c, &g);
            p->E = Tn - k;
        }
    }
}

/* Primary particle for the current history: point source at distance SAD
   from the isocentre, uniform over the field rectangle in the isocentre plane
   (Sec. 3), flown to the phantom surface.  Returns 0 if it misses. */
static int make_primary(tctx *c, const or_source *src, part *p) {
    const or_phantom *ph = c->ph;
    double g = src->gantry_deg * PI / 180.0;
    double ax[3] = {sin(g), 0.0, cos(g)}, e1[3] = {cos(g), 0.0, -sin(g)}, e2[3] = {0, 1, 0};
    double S[3], P[3];
    double a = (ranecu_next(&c->rng) - 0.5) * src->fx, b = (ranecu_next(&c->rng) - 0.5) * src->fy;
    for (int i = 0; i < 3; i++) {
        S[i] = src->iso[i] - src->sad * ax[i];
        P[i] = src->iso[i] + a * e1[i] + b * e2[i];
    }
    double d[3] = {P[0] - S[0], P[1] - S[1], P[2] - S[2]};
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; i++) d[i] /= n;
    p->E = src->spectrum == 1 ? sample_spectrum(&c->rng) : src->energy;
    p->type = src->particle == 0 ? 0 : 1;
    /* slab-method ray/box intersection */
    const double L[3] = {ph->nx * ph->dx, ph->ny * ph->dy, ph->nz * ph->dz};
    const double D[3] = {ph->dx, ph->dy, ph->dz};
    const int N[3] = {ph->nx, ph->ny, ph->nz};
    double t0 = 0.0, t1 = INF;
    int face = -1;
    for (int i = 0; i < 3; i++) {
        if (d[i] == 0.0) {
            if (S[i] < 0 || S[i] > L[i]) return 0;
            continue;
        }
        double ta = (0.0 - S[i]) / d[i], tb = (L[i] - S[i]) / d[i];
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t0) { t0 = ta; face = i; }
        if (tb < t1) t1 = tb;
    }
    if (!(t1 > t0)) return 0;
    for (int i = 0; i < 3; i++) {
        p->x[i] = S[i] + t0 * d[i];
        p->d[i] = d[i];
    }
    if (face >= 0) p->x[face] = d[face] > 0 ? 0.0 : L[face];
    for (int i = 0; i < 3; i++) {
        int k = (int)floor(p->x[i] / D[i]);
        if (k < 0) k = 0;
        if (k > N[i] - 1) k = N[i] - 1;
        p->iv[i] = k;
    }
    return 1;
}

static void tctx_init(tctx *c, const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
                      or_stats *st) {
    memset(c, 0, sizeof(*c));
    c->ph = ph;
    c->mats = mats;
    c->n_mat = n_mat;
    c->p = p;
    c->st = st;
    long V = (long)ph->nx * ph->ny * ph->nz;
    c->hE = (double *)calloc(V, sizeof(double));
    c->cap_touched = 1024;
    c->touched = (long *)malloc(sizeof(long) * c->cap_touched);
    gl_init();
}

static void tctx_free(tctx *c) {
    free(c->hE);
    free(c->touched);
}

int or_run(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p, const or_source *src,
           uint64_t h_begin, uint64_t h_end, uint64_t seed, double *S1, double *S2, or_stats *st) {
    return or_run_planes(ph, mats, n_mat, p, src, h_begin, h_end, seed, S1, S2, NULL, st);
}

/* or_run, plus (if P2 is not NULL) the history-by-history second moment of
   the energy deposited in each z plane: P2[k] += (sum over the plane's voxels
   of the history's deposits)^2, for the exact variance of depth-dose
   integrals (Sec. 3's sigma_D, applied to a plane instead of a voxel). */
int or_run_planes(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
                  const or_source *src, uint64_t h_begin, uint64_t h_end, uint64_t seed, double *S1, double *S2,
                  double *P2, or_stats *st) {
    if (n_mat > OR_MAXMAT) return -1;
    memset(st, 0, sizeof(*st));
    const long nxy = (long)ph->nx * ph->ny;
    double *plane = P2 ? (double *)calloc((size_t)ph->nz, sizeof(double)) : NULL;
    tctx *c = (tctx *)malloc(sizeof(tctx));
    tctx_init(c, ph, mats, n_mat, p, st);
    for (uint64_t h = h_begin; h < h_end; h++) {
        ranecu_seed(&c->rng, seed, h);
        c->h_dep = c->h_esc = 0;
        c->sp = 0;
        part pr;
        st->n_hist++;
        int hit = make_primary(c, src, &pr);
        double emitted = pr.E;
        st->emitted += emitted;
        if (!hit) {
            st->missed += emitted;
            st->n_missed++;
            continue;
        }
        c->stack[c->sp++] = pr;
        while (c->sp > 0 && !c->err) {
            part q = c->stack[--c->sp];
            c->last_v = -1;
            if (q.type == 0) transport_photon(c, &q, 0);
            else transport_electron(c, &q);
        }
        for (long i = 0; i < c->n_touched; i++) {
            long v = c->touched[i];
            double e = c->hE[v];
            S1[v] += e;
            S2[v] += e * e;
            if (plane) plane[v / nxy] += e;
            c->hE[v] = 0.0;
        }
        if (plane) {
            for (long i = 0; i < c->n_touched; i++) {
                long k = c->touched[i] / nxy;
                if (plane[k] != 0.0) {
                    P2[k] += plane[k] * plane[k];
                    plane[k] = 0.0;
                }
            }
        }
        c->n_touched = 0;
        st->deposited += c->h_dep;
        st->deposited2 += c->h_dep * c->h_dep;
        st->escaped += c->h_esc;
        double rel = fabs(emitted - c->h_dep - c->h_esc) / emitted;
        if (rel > st->max_balance_rel) st->max_balance_rel = rel;
    }
    int err = c->err;
    tctx_free(c);
    free(c);
    free(plane);
    return err ? -2 : 0;
}

long long or_uncollided(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
                        const or_source *src, uint64_t n, uint64_t seed) {
    or_stats st;
    memset(&st, 0, sizeof(st));
    tctx *c = (tctx *)malloc(sizeof(tctx));
    tctx_init(c, ph, mats, n_mat, p, &st);
    long long out = 0;
    for (uint64_t h = 0; h < n; h++) {
        ranecu_seed(&c->rng, seed, h);
        part pr;
        if (!make_primary(c, src, &pr)) continue;
        pr.type = 0;
        out += transport_photon(c, &pr, 1);
        for (long i = 0; i < c->n_touched; i++) c->hE[c->touched[i]] = 0.0;
        c->n_touched = 0;
    }
    tctx_free(c);
    free(c);
    return out;
}
