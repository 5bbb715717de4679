// dpm_capi.cu -- the C ABI declared in include/dpm.h: context, device memory,
// phantom upload, table upload, run orchestration (zero slabs -> transport ->
// fold) and result read-back.  The run sequence follows Sec. 2.2: data are
// loaded once, histories are transported in launches, and the dose is copied
// back at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "dpm_ctx.h"
#include "dpm_internal.h"
#include "dpm_kernels.h"
#include "dpm_queue.h"

using namespace dpm;

namespace {

void drop_events(PhantomState *p) {
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  p->folded_transport_ms = p->folded_fold_ms = 0;
  p->folded_launches = 0;
}

// Retire the older half of a phantom's run events into host sums (waits for
// those runs only).
void fold_old_events(PhantomState *p) {
  const size_t n = (p->ev.size() / 6) * 3;
  if (n == 0) return;
  cudaEventSynchronize(p->ev[n - 1]);
  for (size_t i = 0; i + 2 < n; i += 3) {
    float a = 0, b = 0;
    if (cudaEventElapsedTime(&a, p->ev[i], p->ev[i + 1]) == cudaSuccess) p->folded_transport_ms += a;
    if (cudaEventElapsedTime(&b, p->ev[i + 1], p->ev[i + 2]) == cudaSuccess) p->folded_fold_ms += b;
    p->folded_launches++;
  }
  for (size_t i = 0; i < n; ++i) cudaEventDestroy(p->ev[i]);
  p->ev.erase(p->ev.begin(), p->ev.begin() + long(n));
  cudaGetLastError();
}

int fail(dpm_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

#define CUDA_TRY(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(ctx, DPM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// Device allocation owned by the context, counted against its budget.
template <class T>
int dalloc(dpm_ctx *c, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  const size_t bytes = n * sizeof(T);
  if (c->budget && c->in_use + bytes > c->budget)
    return fail(c, DPM_ENOMEM, "device-memory budget of the context exceeded (" + std::to_string(c->in_use) +
                                   " bytes in use, " + std::to_string(bytes) + " more asked, budget " +
                                   std::to_string(c->budget) + ")");
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, DPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->alloc_bytes[*p] = bytes;
  c->in_use += bytes;
  return DPM_OK;
}

// Free a context allocation made by dalloc (NULL is ignored).
void dfree(dpm_ctx *c, void *p) {
  if (!p) return;
  auto it = c->alloc_bytes.find(p);
  if (it != c->alloc_bytes.end()) {
    c->in_use -= it->second;
    c->alloc_bytes.erase(it);
  }
  cudaFree(p);
}

void free_phantom(dpm_ctx *c, PhantomState *p) {
  if (!p) return;
  drop_events(p);
  for (void *d : {(void *)p->d_mat, (void *)p->d_rho, (void *)p->d_mumax, (void *)p->d_mumax64, (void *)p->d_slabs,
                  (void *)p->d_fslabs,
                  (void *)p->d_S1, (void *)p->d_Q, (void *)p->d_counters, (void *)p->d_inv_nb, (void *)p->d_dose,
                  (void *)p->d_sigma, (void *)p->d_dmax})
    dfree(c, d);
}

void free_tables(dpm_ctx *c) {
  for (void *p : c->table_mem) dfree(c, p);
  c->table_mem.clear();
  c->tables_ready = false;
}

PhantomState *get_phantom(dpm_ctx *c, int id) {
  if (id < 0 || id >= int(c->phantoms.size())) return nullptr;
  return c->phantoms[id].get();
}

template <class T>
int upload(dpm_ctx *c, const std::vector<T> &h, const T **out) {
  T *d = nullptr;
  int rc = dalloc(c, &d, h.size());
  if (rc) return rc;
  c->table_mem.push_back(d);
  CUDA_TRY(c, cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = d;
  return DPM_OK;
}

// Photon majorant of a phantom: for every energy node, the largest
// rho * mu/rho over the materials present, at their largest density.
int update_mumax(dpm_ctx *c, PhantomState *p) {
  if (p->mumax_version == c->tables_version || !c->tables_ready) return DPM_OK;
  const HostTables &t = c->ht;
  std::vector<float> mm(t.n_e, 0.f);
  for (int i = 0; i < t.n_e; ++i) {
    double best = 0;
    for (int m = 0; m <= p->max_mat && m < t.n_mat; ++m)
      if (p->rho_max[m] > 0) best = std::max(best, p->rho_max[m] * t.mu_mass_nodes[size_t(m) * t.n_e + i]);
    mm[i] = float(best * (1.0 + 1e-5));
  }
  CUDA_TRY(c, cudaMemcpy(p->d_mumax, mm.data(), mm.size() * sizeof(float), cudaMemcpyHostToDevice));
  p->mumax_version = c->tables_version;
  return DPM_OK;
}

// The same majorant in FP64 (for the FP64 kernel), made on first use.
int update_mumax64(dpm_ctx *c, PhantomState *p) {
  if (p->mumax64_version == c->tables_version) return DPM_OK;
  const HostTables &t = c->ht;
  if (!p->d_mumax64) {
    const int rc = dalloc(c, &p->d_mumax64, size_t(kMaxTableNodes));
    if (rc) return rc;
  }
  std::vector<double> mm(t.n_e, 0.0);
  for (int i = 0; i < t.n_e; ++i) {
    double best = 0;
    for (int m = 0; m <= p->max_mat && m < t.n_mat; ++m)
      if (p->rho_max[m] > 0) best = std::max(best, p->rho_max[m] * t.mu_mass_nodes[size_t(m) * t.n_e + i]);
    mm[i] = best * (1.0 + 1e-5);
  }
  CUDA_TRY(c, cudaMemcpy(p->d_mumax64, mm.data(), mm.size() * sizeof(double), cudaMemcpyHostToDevice));
  p->mumax64_version = c->tables_version;
  return DPM_OK;
}

uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

namespace dpm {

int ctx_fail(dpm_ctx *c, int code, const std::string &msg) { return fail(c, code, msg); }

int ctx_alloc(dpm_ctx *c, void **p, size_t bytes) { return dalloc(c, reinterpret_cast<char **>(p), bytes); }

int ctx_prepare_batches(dpm_ctx *c, PhantomState *p, uint64_t n, int n_batches, uint64_t &bs, int &B) {
  int nb = n_batches > 0 ? n_batches : 50;
  if (nb > 1024) return fail(c, DPM_EINVAL, "n_batches must be <= 1024");
  if (uint64_t(nb) > n) nb = int(n);
  bs = (n + nb - 1) / nb;
  B = int((n + bs - 1) / bs);
  int rc;
  if (p->slab_batches < size_t(B)) {
    dfree(c, p->d_slabs);
    p->d_slabs = nullptr;
    p->slab_batches = 0;
    if ((rc = dalloc(c, &p->d_slabs, size_t(B) * p->V))) return rc;
    p->slab_batches = size_t(B);
  }
  std::vector<double> inv_nb(B);
  for (int b = 0; b < B; ++b) inv_nb[b] = 1.0 / double(std::min<uint64_t>(bs, n - uint64_t(b) * bs));
  CUDA_TRY(c, cudaMemcpyAsync(p->d_inv_nb, inv_nb.data(), B * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  // pageable source: the copy is staged before the call returns
  return DPM_OK;
}

PhantomState *ctx_phantom(dpm_ctx *c, int id) { return get_phantom(c, id); }

template <class Real>
static int fill_run_params(dpm_ctx *c, PhantomState *p, const dpm_source *src, uint64_t first, uint64_t n,
                           uint64_t seed, int physics_flags, const DevTablesT<Real> &tables, const Real *mu_max,
                           RunParamsT<Real> &R) {
  if (!src) return fail(c, DPM_EINVAL, "null source");
  if (!c->tables_ready) return fail(c, DPM_ESTATE, "dpm_build_tables() must precede dpm_run()");
  if (p->max_mat >= c->ht.n_mat) return fail(c, DPM_EINVAL, "phantom uses a material index beyond the tables");
  if (p->mumax_version != c->tables_version) return fail(c, DPM_ESTATE, "photon majorant is stale");
  if (src->particle != 0 && src->particle != 1) return fail(c, DPM_EINVAL, "particle must be 0 or 1");
  if (src->spectrum != 0 && src->spectrum != 1) return fail(c, DPM_EINVAL, "spectrum must be 0 or 1");
  const double emax = src->spectrum == 1 ? 6.0 : src->energy;
  if (!(emax > 0) || emax > c->params.e_max) return fail(c, DPM_EINVAL, "source energy outside (0, e_max]");
  if (!(src->sad > 0) || !(src->fx >= 0) || !(src->fy >= 0)) return fail(c, DPM_EINVAL, "bad beam geometry");
  if (n > 0xFFFFFFFFull) return fail(c, DPM_EINVAL, "at most 2^32-1 histories per call");
  if (physics_flags & ~(DPM_NO_HARD | DPM_NO_MSC | DPM_SAUTER)) return fail(c, DPM_EINVAL, "unknown physics flag");
  R.T = tables;
  R.T.flags = physics_flags;
  R.P.nx = p->nx;
  R.P.ny = p->ny;
  R.P.nz = p->nz;
  R.P.dx = Real(p->dx);
  R.P.dy = Real(p->dy);
  R.P.dz = Real(p->dz);
  R.P.mat = p->d_mat;
  R.P.rho = p->d_rho;
  R.P.mu_max = mu_max;
  const double g = src->gantry_deg * 3.14159265358979323846 / 180.0;
  const double ax[3] = {std::sin(g), 0.0, std::cos(g)};
  R.S.particle = src->particle;
  R.S.spectrum = src->spectrum;
  R.S.energy = Real(src->energy);
  R.S.sx = Real(src->iso[0] - src->sad * ax[0]);
  R.S.sy = Real(src->iso[1] - src->sad * ax[1]);
  R.S.sz = Real(src->iso[2] - src->sad * ax[2]);
  R.S.cx = Real(src->iso[0]);
  R.S.cy = Real(src->iso[1]);
  R.S.cz = Real(src->iso[2]);
  R.S.e1x = Real(std::cos(g));
  R.S.e1z = Real(-std::sin(g));
  R.S.fx = Real(src->fx);
  R.S.fy = Real(src->fy);
  R.first = first;
  R.n = n;
  const uint64_t k = splitmix(seed);
  R.key0 = uint32_t(k);
  R.key1 = uint32_t(k >> 32);
  return DPM_OK;
}

int ctx_run_params(dpm_ctx *c, PhantomState *p, const dpm_source *src, uint64_t first, uint64_t n, uint64_t seed,
                   int physics_flags, RunParams &R) {
  return fill_run_params(c, p, src, first, n, seed, physics_flags, c->dt, (const float *)p->d_mumax, R);
}

int ctx_run_params_f64(dpm_ctx *c, PhantomState *p, const dpm_source *src, uint64_t first, uint64_t n,
                       uint64_t seed, int physics_flags, RunParamsT<double> &R) {
  if (c->tables_ready) {
    const int rc = update_mumax64(c, p);
    if (rc) return rc;
  }
  return fill_run_params(c, p, src, first, n, seed, physics_flags, c->dt64, (const double *)p->d_mumax64, R);
}

}  // namespace dpm

extern "C" {

int dpm_create(dpm_ctx **out, int cuda_device, uint64_t hbm_budget_bytes) {
  if (!out) return DPM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
    cudaGetLastError();
    return DPM_ECUDA;
  }
  dpm_ctx *c = new (std::nothrow) dpm_ctx();
  if (!c) return DPM_ENOMEM;
  c->device = cuda_device;
  c->budget = hbm_budget_bytes;
  c->queue.budget = hbm_budget_bytes;
  c->queue.in_use = &c->in_use;
  if (cudaSetDevice(cuda_device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return DPM_ECUDA;
  }
  c->stream = c->own;
  // load the no-allocation entry point's scratch and the queue kernels now,
  // so that dpm_run_noalloc() finds them resident
  std::string err;
  if (noalloc_setup(err) != DPM_OK) {
    dpm_destroy(c);
    return DPM_ECUDA;
  }
  *out = c;
  return DPM_OK;
}

void dpm_destroy(dpm_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto &p : c->phantoms) free_phantom(c, p.get());
  free_tables(c);
  queue_free(c->queue);
  dfree(c, c->d_jobs);
  dfree(c, c->d_dmax_out);
  dfree(c, c->d_batch_counters);
  for (cudaEvent_t e : c->batch_ev) cudaEventDestroy(e);
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  cudaFree(c->d_err);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

const char *dpm_last_error(const dpm_ctx *c) { return c ? c->err.c_str() : "null context"; }

int dpm_device_bytes(const dpm_ctx *c, uint64_t *in_use, uint64_t *budget) {
  if (!c) return DPM_EINVAL;
  if (in_use) *in_use = c->in_use;
  if (budget) *budget = c->budget;
  return DPM_OK;
}

int dpm_set_stream(dpm_ctx *c, void *s) {
  if (!c) return DPM_EINVAL;
  cudaSetDevice(c->device);
  // the queues, counters and error word are shared by all runs of the context
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, DPM_ECUDA, std::string("previous stream: ") + cudaGetErrorString(e));
  c->stream = s ? (cudaStream_t)s : c->own;
  return DPM_OK;
}

// Validate a phantom's host arrays; its largest material index and the
// largest density of each material (for the photon majorant).
static int scan_phantom(dpm_ctx *c, const uint8_t *mat, const float *rho, size_t V, int &max_mat,
                        double (&rho_max)[DPM_MAX_MAT]) {
  static_assert((DPM_MAX_MAT & (DPM_MAX_MAT - 1)) == 0, "material mask");
  // one pass without branches: four partial maxima per material, so that
  // neighbouring voxels of one material do not wait on each other's store
  float part[4][DPM_MAX_MAT] = {};
  unsigned bad = 0;
  int mm = 0;
  for (size_t v = 0; v < V; ++v) {
    const unsigned m = mat[v];
    const float r = rho[v];
    bad |= unsigned(m >= DPM_MAX_MAT) | unsigned(!(r > 0.f && r <= FLT_MAX));  // also NaN and +inf
    float &a = part[v & 3][m & (DPM_MAX_MAT - 1)];
    a = std::max(a, r);
    mm = std::max(mm, int(m));
  }
  if (bad) {
    for (size_t v = 0; v < V; ++v) {
      if (mat[v] >= DPM_MAX_MAT) return fail(c, DPM_EINVAL, "material index >= 16");
      if (!(rho[v] > 0.f) || !std::isfinite(rho[v])) return fail(c, DPM_EINVAL, "density must be positive and finite");
    }
  }
  max_mat = mm;
  for (int m = 0; m < DPM_MAX_MAT; ++m)
    rho_max[m] = double(std::max(std::max(part[0][m], part[1][m]), std::max(part[2][m], part[3][m])));
  return DPM_OK;
}

int dpm_load_phantom(dpm_ctx *c, int nx, int ny, int nz, double dx, double dy, double dz, const uint8_t *mat,
                     const float *rho, int *phantom_id) {
  if (!c) return DPM_EINVAL;
  if (!mat || !rho || !phantom_id) return fail(c, DPM_EINVAL, "null pointer");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 2047 || ny > 2047 || nz > 1023)
    return fail(c, DPM_EINVAL, "phantom size out of range (1..2047 x 1..2047 x 1..1023)");
  if (!(dx > 0 && dy > 0 && dz > 0)) return fail(c, DPM_EINVAL, "voxel size must be positive");
  cudaSetDevice(c->device);
  auto p = std::make_unique<PhantomState>();
  p->nx = nx; p->ny = ny; p->nz = nz;
  p->dx = dx; p->dy = dy; p->dz = dz;
  p->V = size_t(nx) * ny * nz;
  int rc;
  if ((rc = scan_phantom(c, mat, rho, p->V, p->max_mat, p->rho_max))) return rc;
  if ((rc = dalloc(c, &p->d_mat, p->V)) || (rc = dalloc(c, &p->d_rho, p->V)) || (rc = dalloc(c, &p->d_S1, p->V)) ||
      (rc = dalloc(c, &p->d_Q, p->V)) || (rc = dalloc(c, &p->d_counters, size_t(kCounterSlots))) ||
      (rc = dalloc(c, &p->d_inv_nb, size_t(1024))) || (rc = dalloc(c, &p->d_mumax, size_t(kMaxTableNodes)))) {
    free_phantom(c, p.get());
    return rc;
  }
  CUDA_TRY(c, cudaMemcpyAsync(p->d_mat, mat, p->V, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(p->d_rho, rho, p->V * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_S1, 0, p->V * sizeof(long long), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_Q, 0, p->V * sizeof(double), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_counters, 0, kCounterSlots * sizeof(unsigned long long), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if ((rc = update_mumax(c, p.get()))) {
    free_phantom(c, p.get());
    return rc;
  }
  p->uid = c->next_phantom_uid++;
  c->phantoms.push_back(std::move(p));
  *phantom_id = int(c->phantoms.size()) - 1;
  return DPM_OK;
}

int dpm_free_phantom(dpm_ctx *c, int id) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_phantom(c, p);
  c->phantoms[id].reset();
  return DPM_OK;
}

int dpm_build_tables(dpm_ctx *c, const dpm_material *mats, int n_mat, const dpm_table_params *p) {
  if (!c) return DPM_EINVAL;
  if (!mats || !p) return fail(c, DPM_EINVAL, "null pointer");
  cudaSetDevice(c->device);
  HostTables ht;
  std::string err;
  if (!build_tables(mats, n_mat, *p, ht, err)) return fail(c, DPM_EINVAL, err);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  free_tables(c);
  c->ht = std::move(ht);
  const HostTables &t = c->ht;
  DevTables d{};
  d.n_mat = t.n_mat;
  d.n_e = t.n_e;
  d.lnE_lo = float(std::log(t.e_lo));
  d.inv_dlnE = float((t.n_e - 1) / (std::log(t.e_hi) - std::log(t.e_lo)));
  {
    const double inv = (t.n_e - 1) / (std::log(t.e_hi) - std::log(t.e_lo));
    d.x_lg2 = float(inv * std::log(2.0));
    d.x_lo = float(-std::log(t.e_lo) * inv);
  }
  int rc;
  const float *ph, *el;
  // device layout of the float4 tables: each node's value followed by the
  // float difference to the next node (see el_at in dpm_device.cuh)
  auto with_steps = [&](const auto &h) {
    using T = typename std::decay<decltype(h)>::type::value_type;
    std::vector<T> o(2 * h.size(), T(0));
    for (int m = 0; m < t.n_mat; ++m)
      for (int i = 0; i < t.n_e; ++i)
        for (int k = 0; k < 4; ++k) {
          const size_t at = (size_t(m) * t.n_e + i) * 4 + k;
          o[2 * at - k] = h[at];
          if (i + 1 < t.n_e) {
            volatile T diff = h[at + 4] - h[at];  // one subtraction in the table's type, as on the device
            o[2 * at - k + 4] = diff;
          }
        }
    return o;
  };
  if ((rc = upload(c, with_steps(t.ph), &ph)) || (rc = upload(c, with_steps(t.el), &el)) ||
      (rc = upload(c, t.pmol, &d.pmol)))
    return rc;
  d.ph = reinterpret_cast<const float4 *>(ph);
  d.el = reinterpret_cast<const float4 *>(el);
  auto samp = [&](const std::vector<float> &v, int ne, double lo, double hi, SampTab &s) {
    s.ne = ne;
    s.nu = t.nu;
    s.lnE0 = float(std::log(lo));
    s.inv_dlnE = float((ne - 1) / (std::log(hi) - std::log(lo)));
    return upload(c, v, &s.y);
  };
  if ((rc = samp(t.kn, t.kn_ne, t.kn_lo, t.kn_hi, d.kn)) || (rc = samp(t.mol, t.mol_ne, t.mol_lo, t.mol_hi, d.mol)) ||
      (rc = samp(t.brem, t.brem_ne, t.brem_lo, t.brem_hi, d.brem)) ||
      (rc = samp(t.pair, t.pair_ne, t.pair_lo, t.pair_hi, d.pair)) || (rc = upload(c, t.msc, &d.msc_lnA)) ||
      (rc = samp(t.sauter, t.sauter_ne, t.sauter_lo, t.sauter_hi, d.sauter)))
    return rc;
  d.msc_n = t.msc_n;
  d.msc_x0 = float(t.msc_x0);
  d.msc_inv_dx = float((t.msc_n - 1) / (t.msc_x1 - t.msc_x0));
  d.eabs_e = float(p->eabs_e);
  d.eabs_g = float(p->eabs_g);
  d.wcc = float(p->wcc);
  d.wcr = float(p->wcr);
  d.f_e = float(p->f_e);
  d.x_fe = float(std::log1p(-p->f_e) * (t.n_e - 1) / (std::log(t.e_hi) - std::log(t.e_lo)));
  d.x_eabs = float((std::log(p->eabs_e) - std::log(t.e_lo)) * (t.n_e - 1) / (std::log(t.e_hi) - std::log(t.e_lo)));
  c->dt = d;
  // the FP64 tables for the FP64 kernel
  {
    DevTablesT<double> d64{};
    const double inv = (t.n_e - 1) / (std::log(t.e_hi) - std::log(t.e_lo));
    d64.n_mat = t.n_mat;
    d64.n_e = t.n_e;
    d64.lnE_lo = std::log(t.e_lo);
    d64.inv_dlnE = inv;
    d64.x_lg2 = inv * std::log(2.0);
    d64.x_lo = -std::log(t.e_lo) * inv;
    const double *ph64, *el64;
    if ((rc = upload(c, with_steps(t.ph_64), &ph64)) || (rc = upload(c, with_steps(t.el_64), &el64)) ||
        (rc = upload(c, t.pmol_64, &d64.pmol)))
      return rc;
    d64.ph = reinterpret_cast<const Dbl4 *>(ph64);
    d64.el = reinterpret_cast<const Dbl4 *>(el64);
    auto samp64 = [&](const std::vector<double> &v, int ne, double lo, double hi, SampTabT<double> &s) {
      s.ne = ne;
      s.nu = t.nu;
      s.lnE0 = std::log(lo);
      s.inv_dlnE = (ne - 1) / (std::log(hi) - std::log(lo));
      return upload(c, v, &s.y);
    };
    if ((rc = samp64(t.kn_64, t.kn_ne, t.kn_lo, t.kn_hi, d64.kn)) ||
        (rc = samp64(t.mol_64, t.mol_ne, t.mol_lo, t.mol_hi, d64.mol)) ||
        (rc = samp64(t.brem_64, t.brem_ne, t.brem_lo, t.brem_hi, d64.brem)) ||
        (rc = samp64(t.pair_64, t.pair_ne, t.pair_lo, t.pair_hi, d64.pair)) ||
        (rc = upload(c, t.msc_64, &d64.msc_lnA)) ||
        (rc = samp64(t.sauter_64, t.sauter_ne, t.sauter_lo, t.sauter_hi, d64.sauter)))
      return rc;
    d64.msc_n = t.msc_n;
    d64.msc_x0 = t.msc_x0;
    d64.msc_inv_dx = (t.msc_n - 1) / (t.msc_x1 - t.msc_x0);
    d64.eabs_e = p->eabs_e;
    d64.eabs_g = p->eabs_g;
    d64.wcc = p->wcc;
    d64.wcr = p->wcr;
    d64.f_e = p->f_e;
    d64.x_fe = std::log1p(-p->f_e) * inv;
    d64.x_eabs = (std::log(p->eabs_e) - std::log(t.e_lo)) * inv;
    c->dt64 = d64;
  }
  c->params = *p;
  c->tables_ready = true;
  c->tables_version++;
  for (auto &ph : c->phantoms)
    if (ph && (rc = update_mumax(c, ph.get()))) return rc;
  return DPM_OK;
}

int dpm_clone_phantom(dpm_ctx *c, int src_id, int *phantom_id) {
  if (!c) return DPM_EINVAL;
  PhantomState *s = get_phantom(c, src_id);
  if (!s) return fail(c, DPM_EINVAL, "bad phantom id");
  if (!phantom_id) return fail(c, DPM_EINVAL, "null pointer");
  cudaSetDevice(c->device);
  auto p = std::make_unique<PhantomState>();
  p->nx = s->nx; p->ny = s->ny; p->nz = s->nz;
  p->dx = s->dx; p->dy = s->dy; p->dz = s->dz;
  p->V = s->V;
  p->max_mat = s->max_mat;
  for (int m = 0; m < DPM_MAX_MAT; ++m) p->rho_max[m] = s->rho_max[m];
  int rc;
  if ((rc = dalloc(c, &p->d_mat, p->V)) || (rc = dalloc(c, &p->d_rho, p->V)) || (rc = dalloc(c, &p->d_S1, p->V)) ||
      (rc = dalloc(c, &p->d_Q, p->V)) || (rc = dalloc(c, &p->d_counters, size_t(kCounterSlots))) ||
      (rc = dalloc(c, &p->d_inv_nb, size_t(1024))) || (rc = dalloc(c, &p->d_mumax, size_t(kMaxTableNodes)))) {
    free_phantom(c, p.get());
    return rc;
  }
  // device-to-device, ordered on the context's stream after any pending work
  CUDA_TRY(c, cudaMemcpyAsync(p->d_mat, s->d_mat, p->V, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(p->d_rho, s->d_rho, p->V * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(p->d_mumax, s->d_mumax, kMaxTableNodes * sizeof(float), cudaMemcpyDeviceToDevice,
                              c->stream));
  p->mumax_version = s->mumax_version;
  CUDA_TRY(c, cudaMemsetAsync(p->d_S1, 0, p->V * sizeof(long long), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_Q, 0, p->V * sizeof(double), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_counters, 0, kCounterSlots * sizeof(unsigned long long), c->stream));
  p->uid = c->next_phantom_uid++;
  c->phantoms.push_back(std::move(p));
  *phantom_id = int(c->phantoms.size()) - 1;
  return DPM_OK;
}

int dpm_update_phantom(dpm_ctx *c, int id, const uint8_t *mat, const float *rho) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  if (!mat || !rho) return fail(c, DPM_EINVAL, "null pointer");
  int max_mat = 0;
  double rho_max[DPM_MAX_MAT];
  int rc;
  if ((rc = scan_phantom(c, mat, rho, p->V, max_mat, rho_max))) return rc;
  cudaSetDevice(c->device);
  // earlier runs on the old contents must finish before the copies land
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  p->max_mat = max_mat;
  for (int m = 0; m < DPM_MAX_MAT; ++m) p->rho_max[m] = rho_max[m];
  CUDA_TRY(c, cudaMemcpyAsync(p->d_mat, mat, p->V, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(p->d_rho, rho, p->V * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if ((rc = dpm_reset_tally(c, id))) return rc;
  p->mumax_version = -1;  // new densities: the majorant must be rebuilt
  return update_mumax(c, p);
}

int dpm_reset_tally(dpm_ctx *c, int id) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(p->d_S1, 0, p->V * sizeof(long long), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_Q, 0, p->V * sizeof(double), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(p->d_counters, 0, kCounterSlots * sizeof(unsigned long long), c->stream));
  p->n_total = 0;
  p->b_total = 0;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  drop_events(p);
  return DPM_OK;
}

int dpm_run(dpm_ctx *c, int id, const dpm_source *src, uint64_t first, uint64_t n, uint64_t seed,
            const dpm_run_opts *opts) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  dpm_run_opts o{};
  if (opts) o = *opts;
  if (o.kernel < DPM_KERNEL_QUEUE || o.kernel > DPM_KERNEL_HISTORY_F64)
    return fail(c, DPM_EINVAL, "unknown kernel");
  const bool paper = o.kernel == DPM_KERNEL_PAPER_F32 || o.kernel == DPM_KERNEL_PAPER_CAS;
  const bool f64 = o.kernel == DPM_KERNEL_HISTORY_F64;
  RunParams R{};
  RunParamsT<double> R64{};
  int rc = f64 ? ctx_run_params_f64(c, p, src, first, n, seed, o.physics_flags, R64)
               : ctx_run_params(c, p, src, first, n, seed, o.physics_flags, R);
  if (rc) return rc;
  if (n == 0) return DPM_OK;
  cudaSetDevice(c->device);
  uint64_t bs = 0;
  int B = 0;
  if ((rc = ctx_prepare_batches(c, p, n, o.n_batches, bs, B))) return rc;
  if (paper && p->fslab_batches < size_t(B)) {
    dfree(c, p->d_fslabs);
    p->d_fslabs = nullptr;
    p->fslab_batches = 0;
    if ((rc = dalloc(c, &p->d_fslabs, size_t(B) * p->V))) return rc;
    p->fslab_batches = size_t(B);
  }
  if (paper) CUDA_TRY(c, cudaMemsetAsync(p->d_fslabs, 0, size_t(B) * p->V * sizeof(float), c->stream));
  else CUDA_TRY(c, cudaMemsetAsync(p->d_slabs, 0, size_t(B) * p->V * sizeof(unsigned long long), c->stream));
  R.n_batches = B;
  R.slabs = p->d_slabs;
  R.counters = p->d_counters;
  R.err = c->d_err;

  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) CUDA_TRY(c, cudaEventCreate(&ev[i]));
  if (p->ev.size() + 3 > kMaxPendingEvents) fold_old_events(p);
  for (int i = 0; i < 3; ++i) p->ev.push_back(ev[i]);
  if (f64) {
    R64.n_batches = B;
    R64.slabs = p->d_slabs;
    R64.counters = p->d_counters;
    R64.err = c->d_err;
    CUDA_TRY(c, cudaEventRecord(ev[0], c->stream));
    launch_history_f64(R64, bs, c->sm_count, c->stream);
  } else if (o.kernel == DPM_KERNEL_HISTORY) {
    CUDA_TRY(c, cudaEventRecord(ev[0], c->stream));
    launch_history(R, bs, c->sm_count, o.block_size, c->stream);
  } else if (paper) {
    // the float slabs' rounding into the fixed-point slabs counts as transport
    CUDA_TRY(c, cudaEventRecord(ev[0], c->stream));
    launch_history_paper(R, bs, o.kernel == DPM_KERNEL_PAPER_CAS, p->d_fslabs, size_t(B) * p->V, c->sm_count,
                         c->stream);
  } else {
    std::string qerr;
    // automatic refill pause only on queues of 2^kPauseMinLog2 slots or more
    // (the default capacities are; a small queue_log2 needs every refill)
    dpm_run_opts oq = o;
    if (oq.refill_pause == 0 && oq.queue_log2 > 0 && oq.queue_log2 < kPauseMinLog2) oq.refill_pause = -1;
    int qrc = queue_run(c->queue, R, bs, oq, c->sm_count, c->stream, ev[0], qerr);
    if (qrc) return fail(c, qrc, qerr);
  }
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaEventRecord(ev[1], c->stream));
  launch_fold(p->d_slabs, B, p->V, p->d_inv_nb, p->d_S1, p->d_Q, c->sm_count, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaEventRecord(ev[2], c->stream));
  p->n_total += n;
  p->b_total += uint64_t(B);
  return DPM_OK;
}

int dpm_dmax_sigma(dpm_ctx *c, const int *ids, int n, double *out) {
  if (!c) return DPM_EINVAL;
  if (n < 0 || (n > 0 && (!ids || !out))) return fail(c, DPM_EINVAL, "bad arguments");
  cudaSetDevice(c->device);
  std::vector<PhantomState *> ps(n);
  for (int i = 0; i < n; ++i) {
    ps[i] = get_phantom(c, ids[i]);
    if (!ps[i]) return fail(c, DPM_EINVAL, "bad phantom id");
    if (!ps[i]->d_dmax) {
      int rc = dalloc(c, &ps[i]->d_dmax, size_t(4));
      if (rc) return rc;
    }
  }
  if (n > c->dmax_cap) {
    dfree(c, c->d_dmax_out);
    c->d_dmax_out = nullptr;
    c->dmax_cap = 0;
    int rc = dalloc(c, &c->d_dmax_out, size_t(3) * size_t(n));
    if (rc) return rc;
    c->dmax_cap = n;
  }
  // every request's result lands in one device array: one copy back
  for (int i = 0; i < n; ++i) {
    PhantomState *p = ps[i];
    launch_dmax(p->d_S1, p->d_Q, p->d_rho, p->V, double(p->n_total), double(p->b_total), p->dx * p->dy * p->dz,
                p->d_dmax, c->d_dmax_out + 3 * i, c->sm_count, c->stream);
  }
  CUDA_TRY(c, cudaGetLastError());
  const int src = dpm_sync(c);
  if (src == DPM_ECUDA) return src;
  if (n > 0) CUDA_TRY(c, cudaMemcpy(out, c->d_dmax_out, 3 * sizeof(double) * size_t(n), cudaMemcpyDeviceToHost));
  return src;
}

int dpm_sync(dpm_ctx *c) {
  if (!c) return DPM_EINVAL;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int e = 0;
  CUDA_TRY(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(c, cudaMemset(c->d_err, 0, sizeof(int)));
    if (e & ERR_OVERFLOW) return fail(c, DPM_EQUEUE_OVERFLOW, "particle stack or queue overflow");
    if (e & ERR_TIMEOUT) return fail(c, DPM_ETIMEOUT, "a bounded device wait timed out");
    return fail(c, DPM_ESTEPCAP, "a particle exceeded the step limit");
  }
  return DPM_OK;
}

// Fill the run summary; s1_host (if not NULL) already holds the integer tally.
static int read_common(dpm_ctx *c, PhantomState *p, const int64_t *s1_host, dpm_run_stats *st, int sync_rc) {
  if (st) {
    unsigned long long cnt[kCounterSlots];
    CUDA_TRY(c, cudaMemcpy(cnt, p->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    std::memset(st, 0, sizeof(*st));
    st->n_histories = p->n_total;
    st->n_batches = int32_t(p->b_total);
    // the voxel sum can exceed an int64 of 2^-32 MeV quanta: summed exactly,
    // the high (signed) and low 32-bit halves apart, neither of which can
    // overflow 64 bits below 2^32 voxels (the largest phantom has fewer), then
    // rounded once
    std::vector<long long> s1;
    const int64_t *src = s1_host;
    if (!src) {
      s1.resize(p->V);
      CUDA_TRY(c, cudaMemcpy(s1.data(), p->d_S1, p->V * sizeof(long long), cudaMemcpyDeviceToHost));
      src = reinterpret_cast<const int64_t *>(s1.data());
    }
    int64_t hi = 0;
    uint64_t lo = 0;
    for (size_t v = 0; v < p->V; ++v) {
      hi += src[v] >> 32;  // arithmetic shift: floor(x / 2^32)
      lo += uint64_t(src[v]) & 0xffffffffull;
    }
    const __int128 dep = (__int128)hi * 4294967296 + (__int128)lo;
    st->emitted = double((long long)cnt[C_EMIT]) / kCounterScale;
    st->escaped = double((long long)cnt[C_ESC]) / kCounterScale;
    st->missed = double((long long)cnt[C_MISS]) / kCounterScale;
    st->deposited = double(dep) / kTallyScale;
    st->n_e_steps = cnt[C_ESTEP];
    st->n_g_flights = cnt[C_GFLIGHT];
    st->n_g_interactions = cnt[C_GINT];
    st->n_tally_atomics = cnt[C_ATOM];
    st->n_pushed = cnt[C_PUSH];
    st->n_phase_switches = cnt[C_SWITCH];
    st->transport_ms = p->folded_transport_ms;
    st->fold_ms = p->folded_fold_ms;
    st->n_transport_launches = p->folded_launches;
    for (size_t i = 0; i + 2 < p->ev.size(); i += 3) {
      float a = 0, b = 0;
      if (cudaEventElapsedTime(&a, p->ev[i], p->ev[i + 1]) == cudaSuccess) st->transport_ms += a;
      if (cudaEventElapsedTime(&b, p->ev[i + 1], p->ev[i + 2]) == cudaSuccess) st->fold_ms += b;
      st->n_transport_launches++;
    }
    cudaGetLastError();
    drop_events(p);
    st->error_flags = sync_rc == DPM_OK                ? 0
                      : sync_rc == DPM_EQUEUE_OVERFLOW ? 1
                      : sync_rc == DPM_ESTEPCAP        ? 2
                                                       : 4;
  }
  return DPM_OK;
}

int dpm_read_dose(dpm_ctx *c, int id, double *dose, double *sigma, int64_t *s1_raw, dpm_run_stats *st) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  const int src = dpm_sync(c);
  if (src == DPM_ECUDA) return src;
  std::string keep = c->err;
  if (dose || sigma) {
    int rc;
    if (!p->d_dose && ((rc = dalloc(c, &p->d_dose, p->V)) || (rc = dalloc(c, &p->d_sigma, p->V)))) return rc;
    launch_normalize(p->d_S1, p->d_Q, p->d_rho, p->V, double(p->n_total), double(p->b_total), p->dx * p->dy * p->dz,
                     p->d_dose, p->d_sigma, c->sm_count, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    if (dose) CUDA_TRY(c, cudaMemcpyAsync(dose, p->d_dose, p->V * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (sigma) CUDA_TRY(c, cudaMemcpyAsync(sigma, p->d_sigma, p->V * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  if (s1_raw) CUDA_TRY(c, cudaMemcpyAsync(s1_raw, p->d_S1, p->V * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int rc = read_common(c, p, s1_raw, st, src);
  if (rc) return rc;
  if (src) c->err = keep;
  return src;
}

int dpm_read_dose_device(dpm_ctx *c, int id, double *d_dose, double *d_sigma, dpm_run_stats *st) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = get_phantom(c, id);
  if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
  cudaSetDevice(c->device);
  launch_normalize(p->d_S1, p->d_Q, p->d_rho, p->V, double(p->n_total), double(p->b_total), p->dx * p->dy * p->dz,
                   d_dose, d_sigma, c->sm_count, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  if (!st) return DPM_OK;
  const int src = dpm_sync(c);
  if (src == DPM_ECUDA) return src;
  std::string keep = c->err;
  int rc = read_common(c, p, nullptr, st, src);
  if (rc) return rc;
  if (src) c->err = keep;
  return src;
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
int dpm_diag_table(dpm_ctx *c, int which, int mat, int n, const double *energy, const double *aux, double *out) {
  if (!c) return DPM_EINVAL;
  if (!c->tables_ready) return fail(c, DPM_ESTATE, "no tables");
  if (n < 0 || (n > 0 && (!energy || !out)) || which < 0 || which > 9) return fail(c, DPM_EINVAL, "bad arguments");
  if (which == 8 && n > 0 && !aux) return fail(c, DPM_EINVAL, "aux required");
  DevPhantom P{};
  if (which == 9) {
    PhantomState *p = get_phantom(c, mat);
    if (!p) return fail(c, DPM_EINVAL, "bad phantom id");
    int rc = update_mumax(c, p);
    if (rc) return rc;
    P.mu_max = p->d_mumax;
    mat = 0;
  } else if (mat < 0 || mat >= c->ht.n_mat) {
    return fail(c, DPM_EINVAL, "bad material");
  }
  if (n == 0) return DPM_OK;
  cudaSetDevice(c->device);
  double *d = nullptr;
  int rc = dalloc(c, &d, size_t(3) * n);
  if (rc) return rc;
  cudaMemcpy(d, energy, n * sizeof(double), cudaMemcpyHostToDevice);
  if (aux) cudaMemcpy(d + n, aux, n * sizeof(double), cudaMemcpyHostToDevice);
  launch_diag_table(c->dt, P, which, mat, n, d, d + n, d + 2 * n, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, DPM_ECUDA, cudaGetErrorString(e));
  return DPM_OK;
}

int dpm_diag_sample(dpm_ctx *c, int which, double e, double aux, int n, const double *u, double *out) {
  if (!c) return DPM_EINVAL;
  if (!c->tables_ready) return fail(c, DPM_ESTATE, "no tables");
  if (n < 0 || (n > 0 && (!u || !out)) || which < 0 || which > 9) return fail(c, DPM_EINVAL, "bad arguments");
  if (n == 0) return DPM_OK;
  cudaSetDevice(c->device);
  double *d = nullptr;
  int rc = dalloc(c, &d, size_t(2) * n);
  if (rc) return rc;
  cudaMemcpy(d, u, n * sizeof(double), cudaMemcpyHostToDevice);
  launch_diag_sample(c->dt, which, e, aux, n, d, d + n, c->stream);
  cudaError_t er = cudaStreamSynchronize(c->stream);
  if (er == cudaSuccess) er = cudaMemcpy(out, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
  dfree(c, d);
  if (er != cudaSuccess) return fail(c, DPM_ECUDA, cudaGetErrorString(er));
  return DPM_OK;
}

int dpm_diag_philox(dpm_ctx *c, int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  if (!c) return DPM_EINVAL;
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(c, DPM_EINVAL, "bad arguments");
  if (n == 0) return DPM_OK;
  cudaSetDevice(c->device);
  uint32_t *d = nullptr;
  int rc = dalloc(c, &d, size_t(10) * n);
  if (rc) return rc;
  cudaMemcpy(d, ctr, 4 * n * sizeof(uint32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d + 4 * n, key, 2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice);
  launch_diag_philox(n, d, d + 4 * n, d + 6 * n, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 6 * n, 4 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, DPM_ECUDA, cudaGetErrorString(e));
  return DPM_OK;
}

int dpm_diag_atomic_replay(dpm_ctx *c, const uint32_t *ids, uint64_t n, uint64_t n_vox, double *rate) {
  if (!c) return DPM_EINVAL;
  if (!ids || !rate || n == 0 || n > (1ull << 28) || n_vox == 0 || n_vox > (1ull << 32))
    return fail(c, DPM_EINVAL, "need 1..2^28 ids over 1..2^32 voxels and an output");
  for (uint64_t i = 0; i < n; ++i)
    if (ids[i] >= n_vox) return fail(c, DPM_EINVAL, "voxel id out of range");
  cudaSetDevice(c->device);
  unsigned long long *slab = nullptr;
  uint32_t *d_ids = nullptr;
  int rc;
  if ((rc = dalloc(c, &slab, size_t(n_vox)))) return rc;
  if ((rc = dalloc(c, &d_ids, size_t(n)))) {
    dfree(c, slab);
    return rc;
  }
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  cudaError_t e = cudaMemcpyAsync(d_ids, ids, n * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(slab, 0, n_vox * sizeof(unsigned long long), c->stream);
  const int blocks = c->sm_count * 8;
  if (e == cudaSuccess) {
    launch_atomic_replay(slab, d_ids, n, blocks, c->stream);  // warm-up: slab and ids into L2
    cudaEventRecord(ev[0], c->stream);
    launch_atomic_replay(slab, d_ids, n, blocks, c->stream);
    cudaEventRecord(ev[1], c->stream);
    e = cudaStreamSynchronize(c->stream);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  dfree(c, slab);
  dfree(c, d_ids);
  if (e != cudaSuccess) return fail(c, DPM_ECUDA, cudaGetErrorString(e));
  *rate = double(n) / (ms * 1e-3);
  return DPM_OK;
}

int dpm_diag_l2_peaks(dpm_ctx *c, uint64_t ws_bytes, double *out) {
  if (!c) return DPM_EINVAL;
  if (!out || ws_bytes < (1u << 20) || ws_bytes > (64u << 20) || (ws_bytes & (ws_bytes - 1)))
    return fail(c, DPM_EINVAL, "ws_bytes must be a power of two in [1 MiB, 64 MiB]");
  cudaSetDevice(c->device);
  char *d = nullptr;
  int rc = dalloc(c, &d, size_t(ws_bytes) + 256);
  if (rc) return rc;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) cudaEventCreate(&ev[i]);
  unsigned long long *a = reinterpret_cast<unsigned long long *>(d);
  const uint32_t mask = uint32_t(ws_bytes / 8 - 1);
  const int blocks = c->sm_count * 8;
  const int iters = 256;
  float *sink = reinterpret_cast<float *>(d + ws_bytes);
  const size_t n4 = size_t(ws_bytes) / 16;
  const int passes = 16;
  cudaMemsetAsync(d, 0, size_t(ws_bytes) + 256, c->stream);
  // warm-up (brings the buffer into L2), then one timed launch of each
  launch_l2_atomic(a, mask, iters, blocks, c->stream);
  launch_l2_read(reinterpret_cast<const float4 *>(d), n4, 2, sink, blocks, c->stream);
  cudaEventRecord(ev[0], c->stream);
  launch_l2_atomic(a, mask, iters, blocks, c->stream);
  cudaEventRecord(ev[1], c->stream);
  cudaMemsetAsync(d, 0, size_t(ws_bytes), c->stream);
  launch_l2_read(reinterpret_cast<const float4 *>(d), n4, 2, sink, blocks, c->stream);
  cudaEventRecord(ev[2], c->stream);
  launch_l2_read(reinterpret_cast<const float4 *>(d), n4, passes, sink, blocks, c->stream);
  cudaEventRecord(ev[3], c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  float t_atom = 0.f, t_read = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_atom, ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_read, ev[2], ev[3]);
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, DPM_ECUDA, cudaGetErrorString(e));
  out[0] = double(blocks) * 256.0 * iters / (t_atom * 1e-3);
  out[1] = double(ws_bytes) * passes / (t_read * 1e-3);
  return DPM_OK;
}

}  // extern "C"
