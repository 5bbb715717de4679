// dpm_internal.h -- library-internal types shared by the host table builder,
// the kernels and the C ABI.  Nothing here is part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "dpm.h"

namespace dpm {

constexpr double kMc2 = 0.51099895;        // electron rest energy, MeV (CODATA 2018)
constexpr double kRe = 2.8179403262e-13;   // classical electron radius, cm
constexpr double kAlpha = 7.2973525693e-3; // fine-structure constant
constexpr double kNa = 6.02214076e23;      // Avogadro constant, 1/mol
constexpr double kMeVtoJ = 1.602176634e-13;
constexpr double kTallyScale = 4294967296.0; // 2^32 fixed-point quanta per MeV
// The run's energy counters (emitted, escaped, missed) sum every history's
// energy, so they use a coarser quantum: 2^63 / 2^24 MeV = 5.5e11 MeV, room
// for 2e10 histories of 20 MeV; rounding adds ~3e-8 MeV per event.
constexpr double kCounterScale = 16777216.0;  // 2^24 quanta per MeV
constexpr float kCounterScaleF = 16777216.0f;

// The transport arithmetic is FP32 (Sec. 2.3); an FP64 instantiation of the
// same code, with FP64 tables, is kept to measure what single precision costs.
// Four table values of one node in each precision.
struct alignas(32) Dbl4 {
  double x, y, z, w;
};
template <class Real>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = Dbl4;
};

// One inverse-CDF sampling table: rows on a uniform ln(E) grid, columns on a
// uniform grid in the uniform deviate u; entries are a normalised variable in
// [0, 1] whose meaning depends on the process (see dpm_tables.cpp).
template <class Real>
struct SampTabT {
  const Real *y;  // [ne][nu]
  int ne, nu;
  Real lnE0, inv_dlnE;
};

// Device-side view of the tables.  Per-material arrays are [n_mat][n_e].
template <class Real>
struct DevTablesT {
  using V4 = typename Vec4<Real>::type;
  int n_mat, n_e;
  Real lnE_lo, inv_dlnE;
  Real x_lg2, x_lo;  // grid position = log2(E) * x_lg2 + x_lo
  // per-material tables [n_mat][n_e][2]: the node's value, then its
  // difference to the next node (zero at the last node)
  const V4 *ph;    // {mu/rho total (cm^2/g), Compton fraction, photoelectric fraction, 0}
  const V4 *el;    // {R (g/cm^2), S (MeV cm^2/g), Sigma_hard (cm^2/g), 1/lambda1 (cm^2/g)}
  const Real *pmol;   // Moller fraction of Sigma_hard
  SampTabT<Real> kn, mol, brem, pair;
  const Real *msc_lnA;  // ln A on a uniform grid of logit(q)
  int msc_n;
  Real msc_x0, msc_inv_dx;
  Real eabs_e, eabs_g, wcc, wcr, f_e;
  int flags;  // DPM_NO_HARD / DPM_NO_MSC
  Real x_fe, x_eabs;  // grid-index shift of an energy step (1 - f_e), grid index of eabs_e
  SampTabT<Real> sauter;  // photoelectron angle (option DPM_SAUTER): x/x_max of nu/(A+nu)
};

template <class Real>
struct DevPhantomT {
  int nx, ny, nz;
  Real dx, dy, dz;
  const uint8_t *mat;
  const float *rho;
  const Real *mu_max;  // [n_e] photon majorant, 1/cm, on the tables' energy grid
};

template <class Real>
struct DevSourceT {
  int particle, spectrum;
  Real energy;
  Real sx, sy, sz;        // source point
  Real cx, cy, cz;        // isocentre
  Real e1x, e1z;          // field axis 1 (in the x-z plane); axis 2 is y
  Real fx, fy;
};

using SampTab = SampTabT<float>;
using DevTables = DevTablesT<float>;
using DevPhantom = DevPhantomT<float>;
using DevSource = DevSourceT<float>;

// Counters accumulated per thread and reduced at kernel exit.
enum {
  C_EMIT = 0, C_ESC, C_MISS,          // fixed-point energies (2^-32 MeV)
  C_ESTEP, C_GFLIGHT, C_GINT, C_ATOM, C_PUSH,
  C_N
};
// One more device counter beyond the per-thread ones: grid phase switches of
// the queue kernel (counted by the warp that switches).
constexpr int C_SWITCH = C_N;
constexpr int kCounterSlots = C_N + 1;

enum { ERR_OVERFLOW = 1, ERR_STEPCAP = 2, ERR_TIMEOUT = 4 };

constexpr int kMaxJobs = 1024;  // entries of a batch's job table

// One entry of a batch (dpm_run_batch): a phantom, a beam and a history range,
// with the tally slabs and batch size of that phantom's run.
struct DevJob {
  DevPhantom P;
  DevSource S;
  uint64_t first, n;
  uint32_t key0, key1;
  unsigned long long *slabs;  // [n_batches][V]
  uint64_t batch_size;
  uint64_t V;
};

template <class Real>
struct RunParamsT {
  DevTablesT<Real> T;
  DevPhantomT<Real> P;
  DevSourceT<Real> S;
  uint64_t first, n;       // history range
  uint32_t key0, key1;     // Philox key from the seed
  int n_batches;
  unsigned long long *slabs;  // [n_batches][V]
  unsigned long long *counters;  // [kCounterSlots] (energies as two's-complement int64)
  int *err;
  const DevJob *jobs;  // batch launches only: the job table (global memory)
  int n_jobs;
  int n_photon_jobs;   // the table lists photon-beam jobs first, then electron-beam jobs
};
using RunParams = RunParamsT<float>;

// Host-built tables: the closed forms evaluated in FP64 (the *_64 arrays, for
// the FP64 kernel) and rounded to FP32 (for the transport kernels).
struct HostTables {
  int n_mat = 0, n_e = 0;
  double e_lo = 0, e_hi = 0;
  std::vector<float> ph, el, pmol;
  std::vector<float> kn, mol, brem, pair, msc, sauter;
  std::vector<double> ph_64, el_64, pmol_64;
  std::vector<double> kn_64, mol_64, brem_64, pair_64, msc_64, sauter_64;
  int sauter_ne = 0;
  double sauter_lo = 0, sauter_hi = 0;
  int kn_ne = 0, mol_ne = 0, brem_ne = 0, pair_ne = 0, nu = 0, msc_n = 0;
  double kn_lo = 0, kn_hi = 0, mol_lo = 0, mol_hi = 0, brem_lo = 0, brem_hi = 0, pair_lo = 0, pair_hi = 0;
  double msc_x0 = 0, msc_x1 = 0;
  std::vector<double> mu_mass_nodes;  // [n_mat][n_e] FP64 mu/rho for the majorant
};

bool build_tables(const dpm_material *mats, int n_mat, const dpm_table_params &p, HostTables &out,
                  std::string &err);

}  // namespace dpm
