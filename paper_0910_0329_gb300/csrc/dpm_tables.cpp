// dpm_tables.cpp -- host construction of the device tables.
//
// The transport kernels never evaluate a cross section: everything they need
// is tabulated here once per dpm_build_tables() call, in FP64, and stored as
// FP32 (Sec. 2.3 keeps the paper's data as single-precision tables in texture
// memory; here they are plain arrays read through the L1/L2 caches).
//
// Model (the closed forms this library adopts for DPM's tabulated data,
// Sec. 2.1):
//   photons   Klein-Nishina (free electrons); photoelectric c_pe sum(wZ^4/A)/E^3;
//             unscreened extreme-relativistic Bethe-Heitler pair production
//             with the logarithm clamped at zero;
//   electrons Bethe restricted collision stopping power (ICRU 37 form; with
//             the Sternheimer-Peierls density effect for a material that
//             gives a density for it) + restricted radiative loss of the simplified
//             Bethe-Heitler spectrum (1/(X0 k))(4/3 - 4/3 y + y^2), X0 from
//             Dahl's fit; hard Moller and bremsstrahlung cross sections;
//             screened-Rutherford transport mean free path with Moliere
//             screening.
// Numerical integration here uses composite Simpson rules.
#include <algorithm>
#include <cmath>
#include <functional>

#include "dpm_internal.h"

namespace dpm {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Per-material constants, computed once from the element list.
struct MatModel {
  double electrons_per_g;   // N_A sum(w Z/A)
  double pe_weight;         // sum(w Z^4/A)
  double pair_weight;       // N_A sum(w Z(Z+1)/A)
  double inv_x0;            // 1/X0 in cm^2/g
  double ln_i2;             // ln((I/mc^2)^2)
  // density effect: delta(X) over X = log10(beta gamma) (de_on false: none)
  bool de_on;
  double de_cbar, de_x0, de_x1, de_a;
  int n;
  double atoms_per_g[DPM_MAX_ELEM], Z[DPM_MAX_ELEM];

  explicit MatModel(const dpm_material &m) {
    electrons_per_g = pe_weight = pair_weight = inv_x0 = 0;
    n = m.n_elem;
    for (int e = 0; e < n; ++e) {
      double z = m.Z[e], a = m.A[e], w = m.w[e];
      electrons_per_g += kNa * w * z / a;
      pe_weight += w * z * z * z * z / a;
      pair_weight += kNa * w * z * (z + 1) / a;
      // Dahl's radiation-length fit for one element
      double x0 = 716.4 * a / (z * (z + 1) * std::log(287.0 / std::sqrt(z)));
      inv_x0 += w / x0;
      atoms_per_g[e] = kNa * w / a;
      Z[e] = z;
    }
    double i_mc2 = m.i_ev * 1e-6 / kMc2;
    ln_i2 = 2.0 * std::log(i_mc2);
    // Sternheimer-Peierls general parameters for a condensed medium: the
    // plasma energy 28.816 sqrt(rho Z/A) eV sets Cbar = 2 ln(I/hw_p) + 1; X0
    // and X1 follow from Cbar and I; a joins the cubic to zero at X0
    de_on = m.rho_de > 0.0;
    de_cbar = de_x0 = de_x1 = de_a = 0.0;
    if (de_on) {
      const double hw_p = 28.816 * std::sqrt(m.rho_de * electrons_per_g / kNa);
      de_cbar = 2.0 * std::log(m.i_ev / hw_p) + 1.0;
      if (m.i_ev < 100.0) {
        de_x1 = 2.0;
        de_x0 = de_cbar < 3.681 ? 0.2 : 0.326 * de_cbar - 1.0;
      } else {
        de_x1 = 3.0;
        de_x0 = de_cbar < 5.215 ? 0.2 : 0.326 * de_cbar - 1.5;
      }
      de_a = (de_cbar - 2.0 * std::log(10.0) * de_x0) / std::pow(de_x1 - de_x0, 3.0);
    }
  }
  // delta at (beta gamma)^2 = bg2
  double density_delta(double bg2) const {
    if (!de_on) return 0.0;
    const double x = 0.5 * std::log10(bg2);
    if (x < de_x0) return 0.0;
    const double d = 2.0 * std::log(10.0) * x - de_cbar;
    return x < de_x1 ? d + de_a * std::pow(de_x1 - x, 3.0) : d;
  }
};

double simpson(const std::function<double(double)> &f, double a, double b, int n) {
  if (!(b > a)) return 0.0;
  if (n % 2) ++n;
  double h = (b - a) / n, s = f(a) + f(b);
  for (int i = 1; i < n; ++i) s += f(a + i * h) * ((i & 1) ? 4.0 : 2.0);
  return s * h / 3.0;
}

// ---------------- photons ----------------
double klein_nishina_total(double E) {  // per electron, cm^2
  double k = E / kMc2, a = 1.0 + 2.0 * k, L = std::log(a);
  double bracket = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k) + L / (2.0 * k) - (1.0 + 3.0 * k) / (a * a);
  return 2.0 * kPi * kRe * kRe * bracket;
}

// Antiderivative of the Klein-Nishina eps density up to constants: the density
// (eps + 1/eps - sin^2 theta) with cos theta = 1 + 1/k - 1/(k eps) expands to
// eps + (c^2 - 1) + (1 - 2c/k)/eps + 1/(k^2 eps^2), c = 1 + 1/k.
double kn_prim(double k, double e) {
  double c = 1.0 + 1.0 / k;
  return 0.5 * e * e + (c * c - 1.0) * e + (1.0 - 2.0 * c / k) * std::log(e) - 1.0 / (k * k * e);
}

// Bethe-Heitler pair shape (electron share eps), clamped at zero.
double pair_shape(double k, double e) {
  double l = std::log(2.0 * k * e * (1.0 - e)) - 0.5;
  if (l <= 0) return 0.0;
  return (e * e + (1.0 - e) * (1.0 - e) + (2.0 / 3.0) * e * (1.0 - e)) * l;
}

// Support of the clamped pair shape inside the kinematic range [1/k, 1-1/k].
bool pair_support(double k, double &lo, double &hi) {
  double disc = 1.0 - 2.0 * std::exp(0.5) / k;
  if (k <= 2.0 || disc <= 0) return false;
  double r = std::sqrt(disc);
  lo = std::max(1.0 / k, 0.5 * (1.0 - r));
  hi = std::min(1.0 - 1.0 / k, 0.5 * (1.0 + r));
  return hi > lo;
}

double pair_integral(double k) {  // 4 * integral of the clamped shape
  double lo, hi;
  if (!pair_support(k, lo, hi)) return 0.0;
  return 4.0 * simpson([k](double e) { return pair_shape(k, e); }, lo, hi, 1024);
}

void photon_mu(const MatModel &m, double E, double c_pe, double &mc, double &mpe, double &mpair) {
  mc = m.electrons_per_g * klein_nishina_total(E);
  mpe = c_pe * m.pe_weight / (E * E * E);
  mpair = m.pair_weight * kAlpha * kRe * kRe * pair_integral(E / kMc2);
}

// ---------------- electrons ----------------
struct Kin {
  double tau, gam, beta2, bg2;
  explicit Kin(double T) : tau(T / kMc2), gam(T / kMc2 + 1.0) {
    beta2 = 1.0 - 1.0 / (gam * gam);
    bg2 = tau * (tau + 2.0);
  }
};

double s_collision(const MatModel &m, double T, double wcc) {
  Kin k(T);
  double d = std::min(wcc / kMc2, 0.5 * k.tau);
  double F = -1.0 - k.beta2 + std::log((k.tau - d) * d) + k.tau / (k.tau - d) +
             (0.5 * d * d + (2.0 * k.tau + 1.0) * std::log(1.0 - d / k.tau)) / (k.gam * k.gam);
  double B = std::log(2.0 * (k.tau + 2.0)) - m.ln_i2 + F - m.density_delta(k.bg2);
  return 2.0 * kPi * kRe * kRe * kMc2 * m.electrons_per_g / k.beta2 * B;
}

double s_radiative(const MatModel &m, double T, double wcr) {
  double E = T + kMc2, y = std::min(wcr, T) / E;
  return E * m.inv_x0 * y * (4.0 / 3.0 - y * (2.0 / 3.0 - y / 3.0));
}

double sigma_moller(const MatModel &m, double T, double wcc) {
  if (T <= 2.0 * wcc) return 0.0;
  Kin k(T);
  double ec = wcc / T, a = (k.tau / k.gam) * (k.tau / k.gam), b = (2.0 * k.tau + 1.0) / (k.gam * k.gam);
  double I = (1.0 / ec - 1.0 / (1.0 - ec)) + a * (0.5 - ec) - b * std::log((1.0 - ec) / ec);
  return m.electrons_per_g * 2.0 * kPi * kRe * kRe * kMc2 / (k.beta2 * T) * I;
}

// Antiderivative of the Moller bracket 1/e^2 + 1/(1-e)^2 + a - b/(e(1-e)).
double moller_prim(double a, double b, double e) {
  return -1.0 / e + 1.0 / (1.0 - e) + a * e - b * std::log(e / (1.0 - e));
}

double sigma_brems(const MatModel &m, double T, double wcr) {
  if (T <= wcr) return 0.0;
  double E = T + kMc2;
  return m.inv_x0 * ((4.0 / 3.0) * std::log(T / wcr) - (4.0 / 3.0) * (T - wcr) / E + (T * T - wcr * wcr) / (2.0 * E * E));
}

double brems_prim(double E, double k) {  // antiderivative of (1/k)(4/3 - 4/3 k/E + k^2/E^2)
  return (4.0 / 3.0) * std::log(k) - (4.0 / 3.0) * k / E + 0.5 * k * k / (E * E);
}

double inv_lambda1(const MatModel &m, double T) {
  Kin k(T);
  double s = 0;
  for (int e = 0; e < m.n; ++e) {
    double z = m.Z[e];
    double chi0 = kAlpha * std::cbrt(z) / 0.885;
    double eta = 0.25 * chi0 * chi0 / k.bg2 * (1.13 + 3.76 * (kAlpha * z) * (kAlpha * z) / k.beta2);
    double G = std::log1p(1.0 / eta) - 1.0 / (1.0 + eta);
    s += m.atoms_per_g[e] * 2.0 * kPi * z * (z + 1.0) * kRe * kRe / (k.beta2 * k.bg2) * G;
  }
  return s;
}

// ---------------- inversion helper ----------------
// x in [lo, hi] with F(x) = target for increasing F, by bisection.
double invert(const std::function<double(double)> &F, double lo, double hi, double target) {
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    (F(mid) < target ? lo : hi) = mid;
  }
  return 0.5 * (lo + hi);
}

// mean of (1-mu) for the hinge distribution 2A(1+A)/(x+2A)^2, written as
// 2h/x with h = (1+1/x) ln(1+x) - 1, x = 1/A (series for small x).
double hinge_mean(double A) {
  double x = 1.0 / A;
  double h;
  if (x > 1e-3) {
    h = (1.0 + 1.0 / x) * std::log1p(x) - 1.0;
  } else {
    h = 0;
    double p = x;
    for (int n = 2; n < 12; ++n) {
      h += ((n & 1) ? -1.0 : 1.0) * p / (n * (n - 1.0));
      p *= x;
    }
  }
  return 2.0 * h / x;
}

}  // namespace

bool build_tables(const dpm_material *mats, int n_mat, const dpm_table_params &p, HostTables &t, std::string &err) {
  if (n_mat < 1 || n_mat > DPM_MAX_MAT) { err = "n_mat out of range"; return false; }
  if (p.n_e < 64 || p.n_e > (1 << 16)) { err = "n_e out of range [64, 65536]"; return false; }
  if (!(p.eabs_e > 0 && p.eabs_g > 0 && p.wcc > 0 && p.wcr > 0 && p.f_e > 0 && p.f_e < 1 && p.c_pe >= 0)) {
    err = "invalid transport parameters";
    return false;
  }
  if (!(p.e_max > 2.0 * std::max(p.eabs_e, p.eabs_g))) { err = "e_max too small"; return false; }
  for (int m = 0; m < n_mat; ++m) {
    if (mats[m].n_elem < 1 || mats[m].n_elem > DPM_MAX_ELEM || !(mats[m].i_ev > 0) ||
        !(mats[m].rho_de >= 0 && std::isfinite(mats[m].rho_de))) {
      err = "invalid material " + std::to_string(m);
      return false;
    }
    for (int e = 0; e < mats[m].n_elem; ++e)
      if (!(mats[m].Z[e] >= 1 && mats[m].A[e] > 0 && mats[m].w[e] >= 0)) {
        err = "invalid element in material " + std::to_string(m);
        return false;
      }
  }
  std::vector<MatModel> mm;
  for (int m = 0; m < n_mat; ++m) mm.emplace_back(mats[m]);

  const int N = p.n_e;
  t.n_mat = n_mat;
  t.n_e = N;
  t.e_lo = 0.99 * std::min(p.eabs_e, p.eabs_g);
  t.e_hi = 1.01 * p.e_max;
  const double l0 = std::log(t.e_lo), dl = (std::log(t.e_hi) - l0) / (N - 1);
  auto node_E = [&](int i) { return std::exp(l0 + i * dl); };

  t.ph_64.assign(size_t(n_mat) * N * 4, 0.0);
  t.el_64.assign(size_t(n_mat) * N * 4, 0.0);
  t.pmol_64.assign(size_t(n_mat) * N, 0.0);
  t.mu_mass_nodes.assign(size_t(n_mat) * N, 0.0);

  const double kinks[2] = {std::min(p.wcr, 2.0 * p.wcc), std::max(p.wcr, 2.0 * p.wcc)};
  for (int m = 0; m < n_mat; ++m) {
    const MatModel &M = mm[m];
    auto S = [&](double T) { return s_collision(M, T, p.wcc) + s_radiative(M, T, p.wcr); };
    auto dR = [&](double a, double b) {  // integral of dT/S over [a, b] in u = ln T, split at kinks
      double s = 0, lo = a;
      for (double kk : kinks)
        if (kk > lo && kk < b) {
          s += simpson([&](double u) { double T = std::exp(u); return T / S(T); }, std::log(lo), std::log(kk), 8);
          lo = kk;
        }
      return s + simpson([&](double u) { double T = std::exp(u); return T / S(T); }, std::log(lo), std::log(b), 8);
    };
    double R = 0;
    for (int i = 0; i < N; ++i) {
      double E = node_E(i);
      double mc, mpe, mpair;
      photon_mu(M, E, p.c_pe, mc, mpe, mpair);
      double mt = mc + mpe + mpair;
      size_t o = (size_t(m) * N + i) * 4;
      t.ph_64[o + 0] = mt;
      t.ph_64[o + 1] = mc / mt;
      t.ph_64[o + 2] = mpe / mt;
      t.mu_mass_nodes[size_t(m) * N + i] = mt;
      if (i > 0) R += dR(node_E(i - 1), E);
      double sm = sigma_moller(M, E, p.wcc), sb = sigma_brems(M, E, p.wcr);
      t.el_64[o + 0] = R;
      t.el_64[o + 1] = S(E);
      t.el_64[o + 2] = sm + sb;
      t.el_64[o + 3] = inv_lambda1(M, E);
      t.pmol_64[size_t(m) * N + i] = sm + sb > 0 ? sm / (sm + sb) : 0.0;
    }
  }

  // ---- inverse-CDF sampling tables: rows on ln E, NU columns in u ----
  const int NU = 129, NR = 256;
  t.nu = NU;
  auto row_grid = [&](double lo, double hi, double &glo, double &ghi) { glo = lo; ghi = hi; };

  // Klein-Nishina: y = ln(eps)/ln(eps0), eps0 = 1/(1+2k)
  row_grid(t.e_lo, t.e_hi, t.kn_lo, t.kn_hi);
  t.kn_ne = NR;
  t.kn_64.assign(size_t(NR) * NU, 0.0);
  for (int r = 0; r < NR; ++r) {
    double E = std::exp(std::log(t.kn_lo) + r * (std::log(t.kn_hi) - std::log(t.kn_lo)) / (NR - 1));
    double k = E / kMc2, e0 = 1.0 / (1.0 + 2.0 * k), P0 = kn_prim(k, e0), P1 = kn_prim(k, 1.0);
    for (int c = 0; c < NU; ++c) {
      double u = double(c) / (NU - 1), e;
      if (c == 0) e = e0;
      else if (c == NU - 1) e = 1.0;
      else e = std::exp(invert([&](double le) { return (kn_prim(k, std::exp(le)) - P0) / (P1 - P0); }, std::log(e0), 0.0, u));
      t.kn_64[size_t(r) * NU + c] = std::log(e) / std::log(e0);
    }
  }

  // Moller: z = (1/ec - 1/eps)/(1/ec - 2), eps = W/T in [ec, 1/2], ec = wcc/T
  row_grid(2.0 * p.wcc * 1.0001, t.e_hi, t.mol_lo, t.mol_hi);
  t.mol_ne = NR;
  t.mol_64.assign(size_t(NR) * NU, 0.0);
  for (int r = 0; r < NR; ++r) {
    double T = std::exp(std::log(t.mol_lo) + r * (std::log(t.mol_hi) - std::log(t.mol_lo)) / (NR - 1));
    Kin k(T);
    double ec = p.wcc / T, a = (k.tau / k.gam) * (k.tau / k.gam), b = (2.0 * k.tau + 1.0) / (k.gam * k.gam);
    double P0 = moller_prim(a, b, ec), P1 = moller_prim(a, b, 0.5);
    for (int c = 0; c < NU; ++c) {
      double u = double(c) / (NU - 1), e;
      if (c == 0) e = ec;
      else if (c == NU - 1) e = 0.5;
      else e = invert([&](double x) { return (moller_prim(a, b, x) - P0) / (P1 - P0); }, ec, 0.5, u);
      t.mol_64[size_t(r) * NU + c] = (1.0 / ec - 1.0 / e) / (1.0 / ec - 2.0);
    }
  }

  // bremsstrahlung: y = ln(k/wcr)/ln(T/wcr)
  row_grid(p.wcr * 1.0001, t.e_hi, t.brem_lo, t.brem_hi);
  t.brem_ne = NR;
  t.brem_64.assign(size_t(NR) * NU, 0.0);
  for (int r = 0; r < NR; ++r) {
    double T = std::exp(std::log(t.brem_lo) + r * (std::log(t.brem_hi) - std::log(t.brem_lo)) / (NR - 1));
    double E = T + kMc2, P0 = brems_prim(E, p.wcr), P1 = brems_prim(E, T);
    for (int c = 0; c < NU; ++c) {
      double u = double(c) / (NU - 1), kk;
      if (c == 0) kk = p.wcr;
      else if (c == NU - 1) kk = T;
      else kk = std::exp(invert([&](double lk) { return (brems_prim(E, std::exp(lk)) - P0) / (P1 - P0); },
                                std::log(p.wcr), std::log(T), u));
      t.brem_64[size_t(r) * NU + c] = std::log(kk / p.wcr) / std::log(T / p.wcr);
    }
  }

  // pair: y = (eps - lo)/(hi - lo) on the support of the clamped shape
  row_grid(2.0 * std::exp(0.5) * kMc2 * 1.0001, std::max(t.e_hi, 2.0 * std::exp(0.5) * kMc2 * 1.01), t.pair_lo, t.pair_hi);
  t.pair_ne = NR;
  t.pair_64.assign(size_t(NR) * NU, 0.0);
  {
    const int NF = 4096;
    std::vector<double> cum(NF + 1);
    for (int r = 0; r < NR; ++r) {
      double E = std::exp(std::log(t.pair_lo) + r * (std::log(t.pair_hi) - std::log(t.pair_lo)) / (NR - 1));
      double k = E / kMc2, lo, hi;
      if (!pair_support(k, lo, hi)) {
        for (int c = 0; c < NU; ++c) t.pair_64[size_t(r) * NU + c] = double(c) / (NU - 1);
        continue;
      }
      // cumulative integral on a fine grid (Simpson per cell with the midpoint)
      double h = (hi - lo) / NF;
      cum[0] = 0;
      for (int j = 0; j < NF; ++j) {
        double a = lo + j * h;
        cum[j + 1] = cum[j] + h / 6.0 * (pair_shape(k, a) + 4.0 * pair_shape(k, a + 0.5 * h) + pair_shape(k, a + h));
      }
      for (int c = 0; c < NU; ++c) {
        double target = cum[NF] * double(c) / (NU - 1);
        int j = int(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
        j = std::min(std::max(j, 1), NF);
        double f = (cum[j] > cum[j - 1]) ? (target - cum[j - 1]) / (cum[j] - cum[j - 1]) : 0.0;
        double e = lo + (j - 1 + f) * h;
        t.pair_64[size_t(r) * NU + c] = std::min(1.0, std::max(0.0, (e - lo) / (hi - lo)));
      }
    }
  }

  // Sauter photoelectron angle (option DPM_SAUTER): in x = nu/(A+nu),
  // nu = 1 - cos(theta), A = 1/beta - 1, Sauter's K-shell distribution is
  // p(x) ~ x (2 - (2+A) x) (1 + A B/(1-x)) on [0, 2/(2+A)], B = beta g(g-1)(g-2)/2;
  // y = x / x_max, rows on ln T of the photoelectron, columns uniform in
  // w = acos(1 - 2u)/pi: the density vanishes linearly at both ends of x,
  // so x ~ sqrt(u) and x_max - x ~ sqrt(1-u) there, and in w both ends are
  // linear (a table uniform in u would be steep at the ends)
  row_grid(p.eabs_e, t.e_hi, t.sauter_lo, t.sauter_hi);
  t.sauter_ne = NR;
  t.sauter_64.assign(size_t(NR) * NU, 0.0);
  {
    const int NF = 4096;
    std::vector<double> cum(NF + 1);
    for (int r = 0; r < NR; ++r) {
      const double T = std::exp(std::log(t.sauter_lo) + r * (std::log(t.sauter_hi) - std::log(t.sauter_lo)) / (NR - 1));
      const Kin k(T);
      const double beta = std::sqrt(k.beta2), A = 1.0 / beta - 1.0;
      const double B = 0.5 * beta * k.gam * (k.gam - 1.0) * (k.gam - 2.0);
      const double xm = 2.0 / (2.0 + A);
      auto px = [&](double x) { return x * (2.0 - (2.0 + A) * x) * (1.0 + A * B / (1.0 - x)); };
      const double h = xm / NF;
      cum[0] = 0;
      for (int j = 0; j < NF; ++j) {
        const double a = j * h;
        cum[j + 1] = cum[j] + h / 6.0 * (px(a) + 4.0 * px(a + 0.5 * h) + px(a + h));
      }
      for (int c = 0; c < NU; ++c) {
        const double u = 0.5 * (1.0 - std::cos(kPi * double(c) / (NU - 1)));
        const double target = cum[NF] * u;
        int j = int(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
        j = std::min(std::max(j, 1), NF);
        const double f = (cum[j] > cum[j - 1]) ? (target - cum[j - 1]) / (cum[j] - cum[j - 1]) : 0.0;
        t.sauter_64[size_t(r) * NU + c] = std::min(1.0, std::max(0.0, (j - 1 + f) / NF));
      }
    }
  }

  // multiple scattering: ln A on a uniform grid of x = logit(q)
  t.msc_n = 1025;
  t.msc_x0 = -24.0;
  t.msc_x1 = 24.0;
  t.msc_64.assign(t.msc_n, 0.0);
  for (int i = 0; i < t.msc_n; ++i) {
    double x = t.msc_x0 + i * (t.msc_x1 - t.msc_x0) / (t.msc_n - 1);
    double q = 1.0 / (1.0 + std::exp(-x));
    double lA = invert([&](double la) { return hinge_mean(std::exp(la)); }, -120.0, 80.0, q);
    t.msc_64[i] = lA;
  }
  // the FP32 tables of the transport kernels: each value rounded once
  auto to_f32 = [](const std::vector<double> &d, std::vector<float> &f) {
    f.resize(d.size());
    for (size_t i = 0; i < d.size(); ++i) f[i] = float(d[i]);
  };
  to_f32(t.ph_64, t.ph);
  to_f32(t.el_64, t.el);
  to_f32(t.pmol_64, t.pmol);
  to_f32(t.kn_64, t.kn);
  to_f32(t.mol_64, t.mol);
  to_f32(t.brem_64, t.brem);
  to_f32(t.pair_64, t.pair);
  to_f32(t.msc_64, t.msc);
  to_f32(t.sauter_64, t.sauter);
  return true;
}

}  // namespace dpm
