// dpm_host_tables.cpp -- host-only access to the table builder, so that the
// tables can be inspected on a machine without a GPU (CPU tests of the host
// logic).  Not part of the device path.
#include <cstring>

#include "dpm_host.h"
#include "dpm_internal.h"

extern "C" {

// Build the tables and return a handle (NULL on error, message in err[256]).
void *dpm_host_tables_build(const dpm_material *mats, int n_mat, const dpm_table_params *p, char *err) {
  auto *t = new dpm::HostTables();
  std::string e;
  if (!dpm::build_tables(mats, n_mat, *p, *t, e)) {
    if (err) std::strncpy(err, e.c_str(), 255);
    delete t;
    return nullptr;
  }
  return t;
}

void dpm_host_tables_free(void *h) { delete static_cast<dpm::HostTables *>(h); }

// Copy table `name` into out (at most n floats); returns its length, or -1.
// Scalars are returned through `meta` [e_lo, e_hi, rows, lo, hi, nu].
int dpm_host_tables_get(void *h, const char *name, float *out, int n, double *meta) {
  const dpm::HostTables &t = *static_cast<dpm::HostTables *>(h);
  const std::vector<float> *v = nullptr;
  double m[6] = {t.e_lo, t.e_hi, double(t.n_e), 0, 0, double(t.nu)};
  if (!std::strcmp(name, "ph")) v = &t.ph;
  else if (!std::strcmp(name, "el")) v = &t.el;
  else if (!std::strcmp(name, "pmol")) v = &t.pmol;
  else if (!std::strcmp(name, "kn")) { v = &t.kn; m[2] = t.kn_ne; m[3] = t.kn_lo; m[4] = t.kn_hi; }
  else if (!std::strcmp(name, "mol")) { v = &t.mol; m[2] = t.mol_ne; m[3] = t.mol_lo; m[4] = t.mol_hi; }
  else if (!std::strcmp(name, "brem")) { v = &t.brem; m[2] = t.brem_ne; m[3] = t.brem_lo; m[4] = t.brem_hi; }
  else if (!std::strcmp(name, "pair")) { v = &t.pair; m[2] = t.pair_ne; m[3] = t.pair_lo; m[4] = t.pair_hi; }
  else if (!std::strcmp(name, "msc")) { v = &t.msc; m[2] = t.msc_n; m[3] = t.msc_x0; m[4] = t.msc_x1; }
  else if (!std::strcmp(name, "sauter")) { v = &t.sauter; m[2] = t.sauter_ne; m[3] = t.sauter_lo; m[4] = t.sauter_hi; }
  if (!v) return -1;
  if (meta) std::memcpy(meta, m, sizeof(m));
  if (out) std::memcpy(out, v->data(), sizeof(float) * std::min<size_t>(size_t(n), v->size()));
  return int(v->size());
}
}
