// dpm_batch.cu -- dpm_run_batch(): many (phantom, beam, history range) jobs in
// one persistent queue launch, optionally captured in a CUDA graph, and
// dpm_batch_stats().  The paper runs one problem per program (Sec. 2.2); a
// batch keeps the GPU full across the ends of individual problems.
#include <cuda_runtime.h>

#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "dpm_ctx.h"
#include "dpm_internal.h"
#include "dpm_kernels.h"
#include "dpm_queue.h"

using namespace dpm;

namespace {

#ifndef DPM_SOLO_HISTORIES
#define DPM_SOLO_HISTORIES 3000000
#endif
constexpr uint64_t kSoloHistories = DPM_SOLO_HISTORIES;

#define BATCH_TRY(ctx, call)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return ctx_fail(ctx, DPM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

struct Prepared {
  std::vector<DevJob> tab;       // jobs sharing the persistent launch
  std::vector<PhantomState *> ph;
  std::vector<int> nb;
  std::vector<RunParams> solo;   // jobs too large to share L2 with a neighbour: own launches
  std::vector<PhantomState *> solo_ph;
  std::vector<int> solo_nb;
  std::vector<uint64_t> solo_bs;
  uint64_t total = 0;
};

// Device work of one batch: zero the jobs' slabs, transport (one shared
// persistent launch, then one launch per large job), fold each job.
int batch_device_work(dpm_ctx *c, const Prepared &b, const RunParams &R, const dpm_run_opts &o, int K, int log2cs) {
  for (size_t j = 0; j < b.tab.size(); ++j)
    BATCH_TRY(c, cudaMemsetAsync(b.tab[j].slabs, 0, size_t(b.nb[j]) * b.tab[j].V * sizeof(unsigned long long),
                                 c->stream));
  for (size_t j = 0; j < b.solo.size(); ++j)
    BATCH_TRY(c, cudaMemsetAsync(b.solo[j].slabs, 0, size_t(b.solo_nb[j]) * b.solo_ph[j]->V * sizeof(unsigned long long),
                                 c->stream));
  std::string err;
  int rc;
  // the shared launch pauses refills when its jobs' work is short (the solo
  // launches decide from their own histories)
  dpm_run_opts os = o;
  if (os.refill_pause == 0) {
    double w = 0;
    for (const DevJob &J : b.tab) w += double(J.n) * (J.S.particle == 0 ? 1.0 : kElectronHistoryWeight);
    os.refill_pause = (w <= kPauseMaxHistories && log2cs >= kPauseMinLog2) ? 1 : -1;
  }
  if (!b.tab.empty() && (rc = queue_launch(c->queue.mem, K, log2cs, R, 0, os, c->sm_count, c->stream, nullptr, err)))
    return ctx_fail(c, rc, err);
  dpm_run_opts oo = o;  // the solo launches decide by their own length, on large enough queues
  if (oo.refill_pause == 0 && log2cs < kPauseMinLog2) oo.refill_pause = -1;
  for (size_t j = 0; j < b.solo.size(); ++j)
    if ((rc = queue_launch(c->queue.mem, K, log2cs, b.solo[j], b.solo_bs[j], oo, c->sm_count, c->stream, nullptr, err)))
      return ctx_fail(c, rc, err);
  for (size_t j = 0; j < b.tab.size(); ++j) {
    PhantomState *p = b.ph[j];
    launch_fold(p->d_slabs, b.nb[j], p->V, p->d_inv_nb, p->d_S1, p->d_Q, c->sm_count, c->stream);
  }
  for (size_t j = 0; j < b.solo.size(); ++j) {
    PhantomState *p = b.solo_ph[j];
    launch_fold(p->d_slabs, b.solo_nb[j], p->V, p->d_inv_nb, p->d_S1, p->d_Q, c->sm_count, c->stream);
  }
  BATCH_TRY(c, cudaGetLastError());
  return DPM_OK;
}

}  // namespace

extern "C" int dpm_run_batch(dpm_ctx *c, const dpm_job *jobs, int n_jobs, const dpm_run_opts *opts) {
  if (!c) return DPM_EINVAL;
  if (n_jobs < 0 || n_jobs > kMaxJobs || (n_jobs > 0 && !jobs)) return ctx_fail(c, DPM_EINVAL, "bad job list");
  dpm_run_opts o{};
  if (opts) o = *opts;
  if (o.kernel != DPM_KERNEL_QUEUE) return ctx_fail(c, DPM_EINVAL, "batches run on the queue kernel");
  cudaSetDevice(c->device);
  Prepared b;
  std::set<int> seen;
  int rc;
  // A job gets its own launch (in the same stream or graph) when its phantom
  // and hot tally slab (13 bytes per voxel) exceed a quarter of L2 -- two
  // such jobs overlapping at a job boundary evict each other (13-15 % slower
  // on 256x256x128 phantoms) -- or when it has kSoloHistories or more: the
  // shared launch reads each particle's job record on every step and only
  // gains from filling short jobs' start-up and drain.  With the records in
  // shared memory the 64-job batch measured 741 / 732 / 730 / 731 / 751 ms
  // with the split at 1, 2, 3, 5 and 10 million histories (755 ms as 64
  // separate runs).
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
  const size_t solo_bytes = size_t(l2 > 0 ? l2 : (96 << 20)) / 4;
  for (int j = 0; j < n_jobs; ++j) {
    PhantomState *p = ctx_phantom(c, jobs[j].phantom_id);
    if (!p) return ctx_fail(c, DPM_EINVAL, "bad phantom id in job " + std::to_string(j));
    if (!seen.insert(jobs[j].phantom_id).second) return ctx_fail(c, DPM_EINVAL, "jobs of a batch need distinct phantoms");
    RunParams Rj{};
    if ((rc = ctx_run_params(c, p, &jobs[j].src, jobs[j].first_history, jobs[j].n_histories, jobs[j].seed,
                             o.physics_flags, Rj)))
      return rc;
    if (jobs[j].n_histories == 0) continue;
    if (jobs[j].n_histories > 0x7fffffffull) return ctx_fail(c, DPM_EINVAL, "at most 2^31-1 histories per job");
    uint64_t bs = 0;
    int B = 0;
    if ((rc = ctx_prepare_batches(c, p, jobs[j].n_histories, o.n_batches, bs, B))) return rc;
    b.total += Rj.n;
    // (beyond kSharedJobs small jobs, the rest run on their own as well)
    if (p->V * 13 > solo_bytes || jobs[j].n_histories >= kSoloHistories || int(b.tab.size()) >= kSharedJobs) {
      Rj.n_batches = B;
      Rj.slabs = p->d_slabs;
      Rj.err = c->d_err;
      b.solo.push_back(Rj);
      b.solo_ph.push_back(p);
      b.solo_nb.push_back(B);
      b.solo_bs.push_back(bs);
      continue;
    }
    DevJob J{};
    J.P = Rj.P;
    J.S = Rj.S;
    J.first = Rj.first;
    J.n = Rj.n;
    J.key0 = Rj.key0;
    J.key1 = Rj.key1;
    J.slabs = p->d_slabs;
    J.batch_size = bs;
    J.V = p->V;
    b.tab.push_back(J);
    b.ph.push_back(p);
    b.nb.push_back(B);
  }
  if (b.tab.empty() && b.solo.empty()) return DPM_OK;
  // photon-beam jobs first, then electron beams: consecutive jobs of one beam
  // type let warps keep their particle type across job boundaries
  int n_photon = 0;
  {
    Prepared sorted;
    for (int pass = 0; pass < 2; ++pass)
      for (size_t j = 0; j < b.tab.size(); ++j)
        if ((b.tab[j].S.particle == 0) == (pass == 0)) {
          sorted.tab.push_back(b.tab[j]);
          sorted.ph.push_back(b.ph[j]);
          sorted.nb.push_back(b.nb[j]);
          if (pass == 0) ++n_photon;
        }
    sorted.total = b.total;
    sorted.solo = std::move(b.solo);
    sorted.solo_ph = std::move(b.solo_ph);
    sorted.solo_nb = std::move(b.solo_nb);
    sorted.solo_bs = std::move(b.solo_bs);
    b = std::move(sorted);
  }
  if (!c->d_jobs && (rc = ctx_alloc(c, reinterpret_cast<void **>(&c->d_jobs), kMaxJobs * sizeof(DevJob)))) return rc;
  if (!c->d_batch_counters) {
    if ((rc = ctx_alloc(c, reinterpret_cast<void **>(&c->d_batch_counters), kCounterSlots * sizeof(unsigned long long))))
      return rc;
    BATCH_TRY(c, cudaMemsetAsync(c->d_batch_counters, 0, kCounterSlots * sizeof(unsigned long long), c->stream));
  }
  // the job table is read by the kernel at run time (also on graph replays)
  if (!b.tab.empty())
    BATCH_TRY(c, cudaMemcpyAsync(c->d_jobs, b.tab.data(), b.tab.size() * sizeof(DevJob), cudaMemcpyHostToDevice,
                                 c->stream));
  int K = 0, log2cs = 0;
  std::string err;
  if ((rc = queue_prepare(c->queue, o, c->sm_count, K, log2cs, err))) return ctx_fail(c, rc, err);

  for (RunParams &Rs : b.solo) Rs.counters = c->d_batch_counters;
  RunParams R{};
  R.T = c->dt;
  R.T.flags = o.physics_flags;
  if (!b.tab.empty()) {
    R.P = b.tab[0].P;
    R.S = b.tab[0].S;
  }
  R.n = b.total;
  R.jobs = c->d_jobs;
  R.n_jobs = int(b.tab.size());
  R.n_photon_jobs = n_photon;
  R.counters = c->d_batch_counters;
  R.err = c->d_err;

  if (c->batch_ev.size() + 2 > kMaxPendingEvents) {
    // retire the older half of the pending start/end pairs into host sums
    const size_t n = (c->batch_ev.size() / 4) * 2;
    cudaEventSynchronize(c->batch_ev[n - 1]);
    for (size_t i = 0; i + 1 < n; i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, c->batch_ev[i], c->batch_ev[i + 1]) == cudaSuccess) c->batch_folded_ms += ms;
      c->batch_folded_launches++;
    }
    for (size_t i = 0; i < n; ++i) cudaEventDestroy(c->batch_ev[i]);
    c->batch_ev.erase(c->batch_ev.begin(), c->batch_ev.begin() + long(n));
    cudaGetLastError();
  }
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i) BATCH_TRY(c, cudaEventCreate(&ev[i]));
  c->batch_ev.push_back(ev[0]);
  c->batch_ev.push_back(ev[1]);
  if (o.use_graph) {
    std::vector<uint64_t> sig = {uint64_t(reinterpret_cast<uintptr_t>(c->queue.mem)), uint64_t(K), uint64_t(log2cs),
                                 uint64_t(o.refill_min), uint64_t(o.queue_limit),
                                 uint64_t(o.physics_flags), uint64_t(o.timeout_s * 1e6), uint64_t(b.tab.size()),
                                 uint64_t(b.total)};
    for (size_t j = 0; j < b.tab.size(); ++j) {
      sig.push_back(b.ph[j]->uid);
      sig.push_back(uint64_t(reinterpret_cast<uintptr_t>(b.ph[j]->d_slabs)));
      sig.push_back(b.tab[j].n);
      sig.push_back(uint64_t(b.nb[j]));
    }
    // a large job's parameters are baked into its kernel node: its history
    // range, seed and beam become part of the shape
    for (size_t j = 0; j < b.solo.size(); ++j) {
      const RunParams &Rs = b.solo[j];
      sig.push_back(b.solo_ph[j]->uid);
      sig.push_back(uint64_t(reinterpret_cast<uintptr_t>(Rs.slabs)));
      sig.push_back(Rs.first);
      sig.push_back(Rs.n);
      sig.push_back((uint64_t(Rs.key0) << 32) | Rs.key1);
      sig.push_back(uint64_t(b.solo_nb[j]));
      const uint32_t *sw = reinterpret_cast<const uint32_t *>(&Rs.S);
      for (size_t w = 0; w < sizeof(Rs.S) / 4; ++w) sig.push_back(sw[w]);
    }
    // phantoms enter by uid: a freed phantom's host or device addresses may
    // come back in a new one, whose pointers a stale graph would not hold
    if (!c->batch_exec || sig != c->batch_sig) {
      if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
      c->batch_exec = nullptr;
      cudaGraph_t g = nullptr;
      BATCH_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const int wrc = batch_device_work(c, b, R, o, K, log2cs);
      const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (wrc) {
        if (g) cudaGraphDestroy(g);
        return wrc;
      }
      if (e != cudaSuccess) return ctx_fail(c, DPM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&c->batch_exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        c->batch_exec = nullptr;
        return ctx_fail(c, DPM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
      }
      c->batch_sig = sig;
    }
    BATCH_TRY(c, cudaEventRecord(ev[0], c->stream));
    BATCH_TRY(c, cudaGraphLaunch(c->batch_exec, c->stream));
    BATCH_TRY(c, cudaEventRecord(ev[1], c->stream));
  } else {
    BATCH_TRY(c, cudaEventRecord(ev[0], c->stream));
    if ((rc = batch_device_work(c, b, R, o, K, log2cs))) return rc;
    BATCH_TRY(c, cudaEventRecord(ev[1], c->stream));
  }
  for (size_t j = 0; j < b.tab.size(); ++j) {
    b.ph[j]->n_total += b.tab[j].n;
    b.ph[j]->b_total += uint64_t(b.nb[j]);
  }
  for (size_t j = 0; j < b.solo.size(); ++j) {
    b.solo_ph[j]->n_total += b.solo[j].n;
    b.solo_ph[j]->b_total += uint64_t(b.solo_nb[j]);
  }
  c->batch_histories += b.total;
  return DPM_OK;
}

extern "C" int dpm_batch_stats(dpm_ctx *c, dpm_run_stats *st) {
  if (!c) return DPM_EINVAL;
  if (!st) return ctx_fail(c, DPM_EINVAL, "null stats");
  const int sync_rc = dpm_sync(c);
  if (sync_rc == DPM_ECUDA) return sync_rc;
  const std::string keep = c->err;
  std::memset(st, 0, sizeof(*st));
  st->n_histories = c->batch_histories;
  if (c->d_batch_counters) {
    unsigned long long cnt[kCounterSlots];
    BATCH_TRY(c, cudaMemcpy(cnt, c->d_batch_counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    BATCH_TRY(c, cudaMemset(c->d_batch_counters, 0, sizeof(cnt)));
    st->emitted = double((long long)cnt[C_EMIT]) / kCounterScale;
    st->escaped = double((long long)cnt[C_ESC]) / kCounterScale;
    st->missed = double((long long)cnt[C_MISS]) / kCounterScale;
    st->n_e_steps = cnt[C_ESTEP];
    st->n_g_flights = cnt[C_GFLIGHT];
    st->n_g_interactions = cnt[C_GINT];
    st->n_tally_atomics = cnt[C_ATOM];
    st->n_pushed = cnt[C_PUSH];
    st->n_phase_switches = cnt[C_SWITCH];
  }
  st->transport_ms = c->batch_folded_ms;
  st->n_transport_launches = c->batch_folded_launches;
  c->batch_folded_ms = 0;
  c->batch_folded_launches = 0;
  for (size_t i = 0; i + 1 < c->batch_ev.size(); i += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, c->batch_ev[i], c->batch_ev[i + 1]) == cudaSuccess) st->transport_ms += ms;
    st->n_transport_launches++;
  }
  cudaGetLastError();
  for (cudaEvent_t e : c->batch_ev) cudaEventDestroy(e);
  c->batch_ev.clear();
  c->batch_histories = 0;
  st->error_flags = sync_rc == DPM_OK                ? 0
                    : sync_rc == DPM_EQUEUE_OVERFLOW ? 1
                    : sync_rc == DPM_ESTEPCAP        ? 2
                                                     : 4;
  if (sync_rc) c->err = keep;
  return sync_rc;
}
