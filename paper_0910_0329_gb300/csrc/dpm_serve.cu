// dpm_serve.cu -- dpm_server_*(): dose requests served with continuous
// batching on one context.
//
// A request is a beam on one of the geometries resident in the context (a
// loaded phantom).  Each admitted request owns a tally slot: a device copy of
// its geometry (dpm_clone_phantom) with its own integer tally; slots are
// reused after their request is released, and admission stops at the device
// memory budget.  The server works in rounds.  A round takes the active
// requests oldest first while their next chunks fit the round's history
// budget (younger requests with smaller chunks fill the rest), transports them
// in one dpm_run_batch(), finds each one's D_max and sigma on the device
// (dpm_dmax_sigma) and marks the requests that reached the target relative
// sigma as done.  A request's first round runs first_chunk histories; with
// `adaptive` each later round is sized from the request's own relative sigma r
// after n histories: about n (r / target)^2 are needed in all, so the round
// runs that times `overshoot`, minus n, within [first_chunk, max_chunk].  Round
// sizes, history ranges (consecutive, with the request's own seed) and the
// stop decision depend only on the request's own tally, so its result is the
// same alone or in any mix.  The paper runs one problem per program (Sec.
// 2.2); it has no serving loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <string>
#include <vector>

#include "dpm.h"
#include "dpm_ctx.h"

using namespace dpm;

namespace {

struct Request {
  int geometry = -1;
  dpm_source src{};
  uint64_t seed = 0;
  int state = DPM_REQ_PENDING;
  int slot = -1;
  uint64_t histories = 0;
  uint64_t next_n = 0;
  int rounds = 0;
  double rel_sigma = INFINITY, dose_max = 0.0;
  int dmax_voxel = -1;
};

struct Geometry {
  size_t slot_bytes = 0;
  std::vector<int> free_slots;
};

}  // namespace

struct dpm_server {
  dpm_ctx *ctx = nullptr;
  dpm_serve_opts o{};
  std::vector<Request> req;          // by request id
  std::deque<int> pending;           // ids in submission order
  std::vector<int> active;           // ids in admission order
  std::vector<Geometry> geom;        // by geometry phantom id
  std::vector<int> slot_geometry;    // by phantom id: the geometry a slot copies (-1: not a slot)
  uint64_t used = 0;                 // device bytes held by slots
  dpm_server_info info{};            // counters (the queue lengths are filled on read)
};

namespace {

int srv_fail(dpm_server *s, int code, const std::string &msg) {
  s->ctx->err = msg;
  return code;
}

Geometry &geometry(dpm_server *s, int g) {
  if (size_t(g) >= s->geom.size()) s->geom.resize(size_t(g) + 1);
  return s->geom[size_t(g)];
}

// Device bytes of one slot of geometry g: phantom arrays, tally accumulators,
// the round's batch slabs and the fixed per-phantom buffers.
size_t slot_bytes(dpm_server *s, PhantomState *p) {
  const size_t nb = size_t(s->o.n_batches);
  return p->V * (1 + 4 + 8 + 8 + 8 * nb) + kMaxTableNodes * 4 + 16384;
}

Geometry &sized_geometry(dpm_server *s, int g) {
  Geometry &G = geometry(s, g);
  PhantomState *p = ctx_phantom(s->ctx, g);
  if (!G.slot_bytes && p) G.slot_bytes = slot_bytes(s, p);
  return G;
}

// A slot for geometry g: a released one, else a new device copy if the budget
// allows, after freeing released slots of other geometries if it does not;
// -1 if none (the request waits).
int take_slot(dpm_server *s, int g, int &rc) {
  rc = DPM_OK;
  if (!ctx_phantom(s->ctx, g)) {  // the geometry was freed after the request was submitted
    rc = srv_fail(s, DPM_EINVAL, "a request's geometry is no longer loaded");
    return -1;
  }
  Geometry &G = sized_geometry(s, g);
  if (!G.free_slots.empty()) {
    const int id = G.free_slots.back();
    G.free_slots.pop_back();
    return id;
  }
  const uint64_t budget = s->o.hbm_budget_bytes;
  for (size_t h = 0; budget && h < s->geom.size() && s->used + G.slot_bytes > budget; ++h) {
    Geometry &H = s->geom[h];
    while (!H.free_slots.empty() && s->used + G.slot_bytes > budget) {
      const int id = H.free_slots.back();
      H.free_slots.pop_back();
      if ((rc = dpm_free_phantom(s->ctx, id))) return -1;
      s->slot_geometry[size_t(id)] = -1;
      s->used -= H.slot_bytes;
    }
  }
  if (budget && s->used + G.slot_bytes > budget) return -1;
  int id = -1;
  if ((rc = dpm_clone_phantom(s->ctx, g, &id))) return -1;
  if (size_t(id) >= s->slot_geometry.size()) s->slot_geometry.resize(size_t(id) + 1, -1);
  s->slot_geometry[size_t(id)] = g;
  s->used += G.slot_bytes;
  s->info.peak_slot_bytes = std::max(s->info.peak_slot_bytes, s->used);
  return id;
}

// Options with the defaults filled in; false (and a message) if invalid.
bool normalize(dpm_serve_opts &o, std::string &err) {
  if (!(o.target_rel_sigma > 0 && o.target_rel_sigma < 1)) {
    err = "target_rel_sigma must be in (0, 1)";
    return false;
  }
  if (o.first_chunk == 0) o.first_chunk = 200000;
  if (o.max_chunk == 0) o.max_chunk = 32 * o.first_chunk;
  if (o.max_chunk < o.first_chunk || o.max_chunk > 0x7fffffffull) {
    err = "max_chunk must lie in [first_chunk, 2^31-1]";
    return false;
  }
  if (!(o.overshoot > 0)) o.overshoot = 1.15;
  if (o.round_budget == 0) o.round_budget = 40 * o.first_chunk;
  if (o.n_batches <= 0) o.n_batches = 10;
  if (o.n_batches > 1024) {
    err = "n_batches must be <= 1024";
    return false;
  }
  if (o.max_active <= 0 || o.max_active > 1024) o.max_active = 1024;  // jobs of one dpm_run_batch
  return true;
}

uint64_t next_chunk(const dpm_serve_opts &o, uint64_t histories, double rel_sigma) {
  if (!o.adaptive || !std::isfinite(rel_sigma) || rel_sigma <= 0) return o.first_chunk;
  const double q = rel_sigma / o.target_rel_sigma;
  const double need = double(histories) * q * q * o.overshoot - double(histories);
  return uint64_t(std::min(std::max(need, double(o.first_chunk)), double(o.max_chunk)));
}

// Indexes (oldest first) of the requests of the next round: each with its
// whole next chunk while the chunks fit `budget`; a request that does not fit
// is passed over for younger ones with smaller chunks; the oldest always runs.
int select_round(const uint64_t *next_n, int n, uint64_t budget, int *chosen) {
  int k = 0;
  uint64_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (k > 0 && total + next_n[i] > budget) continue;
    chosen[k++] = i;
    total += next_n[i];
  }
  return k;
}

}  // namespace

extern "C" {

int dpm_server_create(dpm_ctx *ctx, const dpm_serve_opts *opts, dpm_server **out) {
  if (!ctx) return DPM_EINVAL;
  if (!out) {
    ctx->err = "null output";
    return DPM_EINVAL;
  }
  dpm_serve_opts o{};
  if (opts) o = *opts;
  std::string err;
  if (!normalize(o, err)) {
    ctx->err = err;
    return DPM_EINVAL;
  }
  auto *s = new dpm_server;
  s->ctx = ctx;
  s->o = o;
  *out = s;
  return DPM_OK;
}

void dpm_server_destroy(dpm_server *s) {
  if (!s) return;
  // the slots stay loaded phantoms of the context (freed with it)
  delete s;
}

int dpm_server_submit(dpm_server *s, int geometry_id, const dpm_source *src, uint64_t seed, int *request_id) {
  if (!s) return DPM_EINVAL;
  if (!src || !request_id) return srv_fail(s, DPM_EINVAL, "null pointer");
  if (!ctx_phantom(s->ctx, geometry_id)) return srv_fail(s, DPM_EINVAL, "bad geometry id");
  if (size_t(geometry_id) < s->slot_geometry.size() && s->slot_geometry[size_t(geometry_id)] >= 0)
    return srv_fail(s, DPM_EINVAL, "a tally slot is not a geometry");
  Request r;
  r.geometry = geometry_id;
  r.src = *src;
  r.seed = seed;
  s->req.push_back(r);
  *request_id = int(s->req.size()) - 1;
  s->pending.push_back(*request_id);
  return DPM_OK;
}

int dpm_server_round(dpm_server *s, int *n_completed) {
  if (!s) return DPM_EINVAL;
  if (n_completed) *n_completed = 0;
  int rc = DPM_OK;
  // admit in submission order while slots and room allow
  for (auto it = s->pending.begin(); it != s->pending.end() && int(s->active.size()) < s->o.max_active;) {
    Request &r = s->req[size_t(*it)];
    const int slot = take_slot(s, r.geometry, rc);
    if (rc) return rc;
    if (slot < 0) {
      ++it;
      continue;
    }
    r.slot = slot;
    r.state = DPM_REQ_ACTIVE;
    r.next_n = s->o.first_chunk;
    s->active.push_back(*it);
    it = s->pending.erase(it);
  }
  if (s->active.empty()) return DPM_OK;
  s->info.max_active = std::max(s->info.max_active, int(s->active.size()));
  // the oldest requests whose next chunks fit the budget (the oldest always)
  std::vector<uint64_t> want(s->active.size());
  for (size_t i = 0; i < s->active.size(); ++i) want[i] = s->req[size_t(s->active[i])].next_n;
  std::vector<int> pick(s->active.size());
  const int k = select_round(want.data(), int(want.size()), s->o.round_budget, pick.data());
  std::vector<int> chosen(static_cast<size_t>(k));
  for (int i = 0; i < k; ++i) chosen[size_t(i)] = s->active[size_t(pick[size_t(i)])];
  std::vector<dpm_job> jobs(chosen.size());
  std::vector<int> slots(chosen.size());
  for (size_t i = 0; i < chosen.size(); ++i) {
    const Request &r = s->req[size_t(chosen[i])];
    jobs[i].phantom_id = r.slot;
    jobs[i].src = r.src;
    jobs[i].first_history = r.histories;
    jobs[i].n_histories = r.next_n;
    jobs[i].seed = r.seed;
    slots[i] = r.slot;
  }
  dpm_run_opts ro{};
  ro.n_batches = s->o.n_batches;
  if ((rc = dpm_run_batch(s->ctx, jobs.data(), int(jobs.size()), &ro))) return rc;
  std::vector<double> res(3 * chosen.size());
  if ((rc = dpm_dmax_sigma(s->ctx, slots.data(), int(slots.size()), res.data()))) return rc;
  // the round's device status (a queue overflow or a timed-out wait is an
  // error of the round) and release of its timing events
  dpm_run_stats st{};
  if ((rc = dpm_batch_stats(s->ctx, &st))) return rc;
  s->info.gpu_ms += st.transport_ms;
  s->info.n_rounds += 1;
  int done = 0;
  for (size_t i = 0; i < chosen.size(); ++i) {
    Request &r = s->req[size_t(chosen[i])];
    r.rounds += 1;
    r.histories += r.next_n;
    s->info.histories += r.next_n;
    r.dose_max = res[3 * i];
    r.rel_sigma = r.dose_max > 0 ? res[3 * i + 1] / r.dose_max : INFINITY;
    r.dmax_voxel = int(res[3 * i + 2]);
    r.next_n = next_chunk(s->o, r.histories, r.rel_sigma);
    if (r.rel_sigma <= s->o.target_rel_sigma) {
      r.state = DPM_REQ_DONE;
      ++done;
    }
  }
  if (done) {
    s->info.n_completed += uint64_t(done);
    s->info.n_done += done;
    std::vector<int> keep;
    for (int id : s->active)
      if (s->req[size_t(id)].state == DPM_REQ_ACTIVE) keep.push_back(id);
    s->active.swap(keep);
  }
  if (n_completed) *n_completed = done;
  return DPM_OK;
}

int dpm_server_status(dpm_server *s, int request_id, dpm_request_status *out) {
  if (!s) return DPM_EINVAL;
  if (!out || request_id < 0 || size_t(request_id) >= s->req.size()) return srv_fail(s, DPM_EINVAL, "bad request");
  const Request &r = s->req[size_t(request_id)];
  out->state = r.state;
  out->slot = r.slot;
  out->histories = r.histories;
  out->rounds = r.rounds;
  out->rel_sigma = r.rel_sigma;
  out->dose_max = r.dose_max;
  out->dmax_voxel = r.dmax_voxel;
  return DPM_OK;
}

int dpm_server_info_get(dpm_server *s, dpm_server_info *out) {
  if (!s) return DPM_EINVAL;
  if (!out) return srv_fail(s, DPM_EINVAL, "null pointer");
  *out = s->info;
  out->n_pending = int(s->pending.size());
  out->n_active = int(s->active.size());
  out->slot_bytes = s->used;
  return DPM_OK;
}

int dpm_server_slot_bytes(dpm_server *s, int geometry_id, uint64_t *bytes) {
  if (!s) return DPM_EINVAL;
  if (!bytes) return srv_fail(s, DPM_EINVAL, "null pointer");
  if (!ctx_phantom(s->ctx, geometry_id)) return srv_fail(s, DPM_EINVAL, "bad geometry id");
  if (size_t(geometry_id) < s->slot_geometry.size() && s->slot_geometry[size_t(geometry_id)] >= 0)
    return srv_fail(s, DPM_EINVAL, "a tally slot is not a geometry");
  *bytes = sized_geometry(s, geometry_id).slot_bytes;
  return DPM_OK;
}

uint64_t dpm_serve_next_chunk(const dpm_serve_opts *opts, uint64_t histories, double rel_sigma) {
  if (!opts) return 0;
  dpm_serve_opts o = *opts;
  std::string err;
  if (!normalize(o, err)) return 0;
  return next_chunk(o, histories, rel_sigma);
}

int dpm_serve_select(const uint64_t *next_n, int n, uint64_t budget, int *chosen) {
  if (n < 0 || (n > 0 && (!next_n || !chosen))) return -1;
  return select_round(next_n, n, budget, chosen);
}

int dpm_server_release(dpm_server *s, int request_id) {
  if (!s) return DPM_EINVAL;
  if (request_id < 0 || size_t(request_id) >= s->req.size()) return srv_fail(s, DPM_EINVAL, "bad request");
  Request &r = s->req[size_t(request_id)];
  if (r.state != DPM_REQ_DONE) return srv_fail(s, DPM_ESTATE, "only a done request can be released");
  int rc;
  if ((rc = dpm_reset_tally(s->ctx, r.slot))) return rc;
  geometry(s, r.geometry).free_slots.push_back(r.slot);
  r.slot = -1;
  r.state = DPM_REQ_RELEASED;
  s->info.n_done -= 1;
  return DPM_OK;
}

}  // extern "C"
