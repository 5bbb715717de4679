/*
 * dpm_oracle.h -- FP64 single-threaded reference transport (TEST INFRASTRUCTURE).
 *
 * This is the oracle that the GPU library is checked against.  It is test
 * infrastructure only: nothing in the product path may link, load or call it;
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Physics (the closed-form model that stands in for DPM's tabulated data; the
 * paper defers all physics to DPM, Sec. 2.1):
 *   photons   Klein-Nishina Compton, Z^4/E^3 photoelectric, unscreened
 *             Bethe-Heitler pair production; ray-marched voxel by voxel with
 *             the real attenuation (no Woodcock majorant);
 *   electrons condensed history: CSDA with the Bethe restricted collision
 *             stopping power (I per material; optionally with the
 *             Sternheimer-Peierls density effect) plus the
 *             restricted bremsstrahlung loss, random-hinge screened-Rutherford
 *             multiple scattering, hard Moller collisions and hard
 *             bremsstrahlung by delta scattering (Sec. 2.1);
 *   tally     exact history-by-history sum and sum of squares per voxel.
 * Random numbers: RANECU (L'Ecuyer 1988), as named in Sec. 2.4, seeded per
 * history so that results do not depend on how histories are split.
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against closed forms, textbook values, identities or brute force.  The
 * assembled transport is pinned in its limiting cases (uncollided photon
 * attenuation, the straight CSDA electron depth-energy profile against an
 * independent ODE solution), by energy conservation per history, mirror
 * symmetry, history-split invariance and brute-force plane moments.  No
 * published coupled dose distribution exists to compare the full transport
 * with (the paper's figures are not in its text).
 */
#ifndef DPM_ORACLE_H
#define DPM_ORACLE_H
#include <stdint.h>

#define OR_MAX_ELEM 8

typedef struct {
    int n_elem;
    double Z[OR_MAX_ELEM], A[OR_MAX_ELEM], w[OR_MAX_ELEM];
    double i_ev;
    double rho_de;  /* density (g/cm^3) of the density-effect correction; 0: none */
} or_material;

enum { OR_NO_HARD = 1, OR_NO_MSC = 2, OR_NO_SECONDARY_PHOTONS = 4, OR_SAUTER = 8 };

typedef struct {
    double eabs_e, eabs_g, wcc, wcr, f_e, c_pe;
    int flags;
} or_params;

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    const uint8_t *mat;
    const float *rho;
} or_phantom;

typedef struct {
    int particle;  /* 0 photon, 1 electron */
    int spectrum;  /* 0 monoenergetic, 1 synthetic 6 MV */
    double energy;
    double iso[3];
    double sad, fx, fy, gantry_deg;
} or_source;

typedef struct {
    double emitted, deposited, escaped, missed;
    double max_balance_rel;          /* max over histories |emit-dep-esc-miss|/emit */
    double deposited2;               /* sum over histories of (energy deposited in the history)^2 */
    double e_path;                   /* total electron path length, cm */
    long long n_hist, n_missed;
    long long n_e_steps, n_g_interactions, n_g_voxel_steps;
    long long n_dep, n_dep_runs;     /* deposits, and runs of same-voxel deposits per particle */
    long long n_sec_e, n_sec_g, n_positrons;
} or_stats;

/* transport ------------------------------------------------------------- */
int or_run(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
           const or_source *src, uint64_t h_begin, uint64_t h_end, uint64_t seed,
           double *S1, double *S2, or_stats *st);
/* or_run plus, if P2 is not NULL (nz doubles, accumulated), the sum over
   histories of the squared energy each history deposits in each z plane. */
int or_run_planes(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
                  const or_source *src, uint64_t h_begin, uint64_t h_end, uint64_t seed, double *S1, double *S2,
                  double *P2, or_stats *st);

/* Primary photons only: counts those leaving the phantom without any
   interaction (narrow-beam uncollided transmission). */
long long or_uncollided(const or_phantom *ph, const or_material *mats, int n_mat, const or_params *p,
                        const or_source *src, uint64_t n, uint64_t seed);

/* physics: cross sections (per electron, cm^2) and coefficients (cm^2/g) --- */
double or_kn_sigma(double E);
double or_kn_dsde(double E, double eps);
double or_kn_cdf(double E, double eps);
double or_mu_compton(const or_material *m, double E);
double or_mu_photo(const or_material *m, double E, double c_pe);
double or_mu_pair(const or_material *m, double E);
double or_pair_integral(double kappa, double lo, double hi, int clamp);
double or_pair_dsde_shape(double kappa, double eps, int clamp);
double or_gl_integrate_test(int which, double a, double b);

/* electrons: stopping powers (MeV cm^2/g), hard cross sections (cm^2/g) --- */
double or_x0(const or_material *m);
double or_scol(const or_material *m, double T, double wcc);
double or_plasma_energy_ev(const or_material *m);
double or_density_delta(const or_material *m, double T);
double or_srad(const or_material *m, double T, double wcr);
double or_moller_sigma(const or_material *m, double T, double wcc);
double or_moller_dsdw(const or_material *m, double T, double W);
double or_brems_sigma(const or_material *m, double T, double wcr);
double or_brems_dsdk(const or_material *m, double T, double k);
double or_lambda1_inv(const or_material *m, double T);
double or_csda_path(const or_material *m, const or_params *p, double T_lo, double T_hi);
double or_csda_energy(const or_material *m, const or_params *p, double T, double mass_path);
double or_msc_A(double q);
double or_msc_mean(double A);
double or_spectrum_cdf(double E);

/* samplers (n draws into out[], RANECU seeded from seed) ------------------ */
void or_sample(int which, double a, double b, const or_material *m, uint64_t n, uint64_t seed, double *out);
enum { OR_S_KN = 0, OR_S_MOLLER = 1, OR_S_BREMS = 2, OR_S_PAIR = 3, OR_S_MSC = 4, OR_S_SPECTRUM = 5, OR_S_SAUTER = 6,
       OR_S_ISO_X = 7, OR_S_ISO_Z = 8 /* x and z of the annihilation photons' isotropic direction */ };

/* One interaction's outgoing particles from direction d_in (pins of the
   kinematics by momentum conservation).  which 0: Compton of a photon of
   energy a into b*a; 1: Moller of an electron of kinetic energy a giving b to
   the secondary.  out = {E1, d1[3], E2, d2[3]}: scattered photon and
   electron, or primary and secondary. */
void or_kinematics(int which, double a, double b, double phi, const double d_in[3], double out[8]);

/* RANECU stream for pins: n uniforms from (s1, s2) */
void or_ranecu_stream(int32_t s1, int32_t s2, int n, double *out, int32_t *state_out);

#endif
