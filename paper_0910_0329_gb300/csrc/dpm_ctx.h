// dpm_ctx.h -- library-internal definition of the context behind the C ABI
// (shared by the translation units that implement ABI calls).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "dpm_internal.h"
#include "dpm_queue.h"

namespace dpm {

constexpr int kMaxTableNodes = 65536;  // upper bound of dpm_table_params.n_e

// Timing events kept per phantom (and per context for batches) between two
// reads of the statistics; past this many the oldest half is waited for,
// its times are summed on the host and its events are released, so that a
// caller that never reads the statistics holds a bounded number of events.
constexpr size_t kMaxPendingEvents = 3 * 1024;

struct PhantomState {
  uint64_t uid = 0;  // unique within the context, never reused (keys the batch graph)
  int nx = 0, ny = 0, nz = 0;
  double dx = 0, dy = 0, dz = 0;
  size_t V = 0;
  uint8_t *d_mat = nullptr;
  float *d_rho = nullptr;
  float *d_mumax = nullptr;  // kMaxTableNodes floats, filled for the current tables
  int mumax_version = -1;
  double *d_mumax64 = nullptr;  // the FP64 majorant (FP64 runs only), n_e doubles
  int mumax64_version = -1;
  int max_mat = 0;
  double rho_max[DPM_MAX_MAT] = {0};
  unsigned long long *d_slabs = nullptr;
  size_t slab_batches = 0;
  float *d_fslabs = nullptr;  // float slabs of the paper's tally (ablation kernels only)
  size_t fslab_batches = 0;
  long long *d_S1 = nullptr;
  double *d_Q = nullptr;
  unsigned long long *d_counters = nullptr;
  double *d_inv_nb = nullptr;
  double *d_dose = nullptr, *d_sigma = nullptr;
  unsigned long long *d_dmax = nullptr;  // [1] key + [3] doubles for the D_max query
  uint64_t n_total = 0;
  uint64_t b_total = 0;
  // CUDA events around each transport launch and fold since the last read;
  // beyond kMaxPendingEvents the oldest runs' times move to the sums below
  std::vector<cudaEvent_t> ev;
  double folded_transport_ms = 0, folded_fold_ms = 0;
  uint64_t folded_launches = 0;
};

}  // namespace dpm

struct dpm_ctx {
  int device = 0;
  // device memory the context keeps (every allocation but the 4-byte error
  // word), against an optional budget (0 = none)
  uint64_t budget = 0, in_use = 0;
  std::unordered_map<const void *, size_t> alloc_bytes;
  int sm_count = 0;
  cudaStream_t own = nullptr, stream = nullptr;
  std::string err;
  bool tables_ready = false;
  int tables_version = 0;
  dpm_table_params params{};
  dpm::HostTables ht;
  dpm::DevTables dt{};
  dpm::DevTablesT<double> dt64{};  // the same tables in FP64 (the FP64 kernel)
  std::vector<void *> table_mem;
  std::vector<std::unique_ptr<dpm::PhantomState>> phantoms;
  uint64_t next_phantom_uid = 1;
  int *d_err = nullptr;
  dpm::QueueState queue;
  // batches
  dpm::DevJob *d_jobs = nullptr;               // job table, kMaxJobs entries
  double *d_dmax_out = nullptr;                // dpm_dmax_sigma results, 3 per phantom [dmax_cap]
  int dmax_cap = 0;
  unsigned long long *d_batch_counters = nullptr;  // [kCounterSlots]
  std::vector<cudaEvent_t> batch_ev;           // start/end pairs since the last dpm_batch_stats
  double batch_folded_ms = 0;                  // times of pairs retired early (see kMaxPendingEvents)
  uint64_t batch_folded_launches = 0;
  uint64_t batch_histories = 0;
  cudaGraphExec_t batch_exec = nullptr;
  std::vector<uint64_t> batch_sig;             // shape the cached graph was captured for
};

namespace dpm {

int ctx_fail(dpm_ctx *c, int code, const std::string &msg);
PhantomState *ctx_phantom(dpm_ctx *c, int id);
// Validate a run request and fill the launch parameters (tally pointers and
// batch size are left to the caller).  Allocates nothing.
int ctx_run_params(dpm_ctx *c, PhantomState *p, const dpm_source *src, uint64_t first, uint64_t n, uint64_t seed,
                   int physics_flags, RunParams &R);
// The same for the FP64 kernel (FP64 tables, source and majorant; builds the
// phantom's FP64 majorant on first use).
int ctx_run_params_f64(dpm_ctx *c, PhantomState *p, const dpm_source *src, uint64_t first, uint64_t n,
                       uint64_t seed, int physics_flags, RunParamsT<double> &R);
// Device allocation owned by the context (error message set on failure).
int ctx_alloc(dpm_ctx *c, void **p, size_t bytes);
// Batch structure of a run of n histories in (at most) n_batches batches:
// makes sure the phantom has B slabs and uploads 1/n_b; returns bs and B.
int ctx_prepare_batches(dpm_ctx *c, PhantomState *p, uint64_t n, int n_batches, uint64_t &bs, int &B);
// With the context's device current: load the module holding the scratch of
// dpm_run_noalloc() and the queue kernels (dpm_noalloc.cu).
int noalloc_setup(std::string &err);

}  // namespace dpm
