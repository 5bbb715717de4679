// dpm_queue.cu -- persistent transport kernel with device-wide particle queues.
//
// The paper runs one history per thread, so the 32 threads of a warp follow
// statistically independent paths and execute mostly one at a time (its
// Sec. 4 diagnosis of the C1060 speed-up).  Here every warp holds particles of
// ONE type (photons or electrons/positrons) in its lanes, steps them together,
// and refills lanes that have finished from per-type particle queues;
// secondaries are pushed to those queues with one atomic per warp.  The
// physics of a particle is the same code as in the per-history kernel and its
// random numbers are keyed by its identity, so both kernels produce the same
// integer tally.
//
// Queues: for each type, one ring per CTA ("shard") in global memory, SoA, with
// a sequence number per slot (a producer publishes position p by writing p+1,
// the consumer frees the slot for position p+capacity), so that producers and
// consumers on different SMs never read a half-written record.  A warp pushes
// to its CTA's shard and pops from it first, stealing from other shards when it
// is empty.  The grid alternates between a source phase and a secondary
// phase (see the scheduler below) so that all SMs run one particle type's
// code at a time.  The run ends when every started warp is idle, every queue
// is empty and the source is exhausted.  Every wait is bounded by a time limit read from
// %globaltimer; on expiry the kernel records an error and returns.
#include <cuda_runtime.h>

#include "dpm_device.cuh"
#include "dpm_queue.h"

namespace dpm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kQBlock = 128;
#ifndef DPM_STEAL_PROBES
#define DPM_STEAL_PROBES 8
#endif
// The whole grid alternates between a source phase (histories start, warps
// track particles of the beam's type) and a secondary phase (no history
// starts, warps track the queued particles of the other type).  The
// secondary phase starts when the other type's particles queued in all
// shards exceed K * (capacity >> HIGH) and ends when they fall below
// K * (capacity >> LOW); photon beams queue electrons, electron beams queue
// bremsstrahlung and annihilation photons.  A CTA whose own shards hold more
// than capacity >> GUARD particles starts no history.
#ifndef DPM_PHASE_HIGH_SHIFT_G
#define DPM_PHASE_HIGH_SHIFT_G 2
#endif
#ifndef DPM_PHASE_LOW_SHIFT_G
#define DPM_PHASE_LOW_SHIFT_G 5
#endif
#ifndef DPM_PHASE_GUARD_SHIFT_G
#define DPM_PHASE_GUARD_SHIFT_G 1
#endif
#ifndef DPM_PHASE_HIGH_SHIFT_E
#define DPM_PHASE_HIGH_SHIFT_E 4
#endif
#ifndef DPM_PHASE_LOW_SHIFT_E
#define DPM_PHASE_LOW_SHIFT_E 7
#endif
#ifndef DPM_PHASE_GUARD_SHIFT_E
#define DPM_PHASE_GUARD_SHIFT_E 2
#endif
constexpr int kStealProbes = DPM_STEAL_PROBES;
// Default refill thresholds (idle lanes) of photon and electron warps.  A
// photon lane's particle is short-lived and starting histories is costly, so
// photon warps gather more idle lanes per refill (6 MV, 10^7 histories:
// 16, 20, 22, 24 and 28 lanes measured 6.65, 6.86, 6.94, 7.01 and 6.99 x 10^8
// histories/s; electron beams within 0.3 % of each other).
#ifndef DPM_REFILL_MIN_G
#define DPM_REFILL_MIN_G 24
#endif
#ifndef DPM_REFILL_MIN_E
#define DPM_REFILL_MIN_E 12
#endif
// Refill pause (kernels with kPause): a warp with particles waits this many
// steps, after a refill that added none, before it tries again.  A failed
// refill costs several dependent L2 round trips (the home shard, then the
// steal probes).  Where the queues have run dry, at the end of a launch, the
// sparse warps that carry the last particles paid that on every step, and
// the end of a launch took longer than its share of histories: a 6 MV launch
// of 10^6 histories takes 2.41 ms without the pause and 2.11 ms with it, one
// of 10^7 1.5 % less time.  In the middle of a long launch the pause costs
// about 1.5 % (6 MV 5x10^7: +1.5 %; 20 MeV electrons at 10^7: +0.7 to
// +0.9 %), so a launch takes it when it is short (queue_launch).  Pauses of
// 8 to 128 steps measured; the longer ones were faster.
#ifndef DPM_REFILL_COOLDOWN
#define DPM_REFILL_COOLDOWN 128
#endif
// Random draws (two Woodcock flights each) a photon lane makes per warp step:
// a warp does not wait for its lane with the longest run of virtual flights.
#ifndef DPM_PHOTON_DRAWS
#define DPM_PHOTON_DRAWS 1
#endif
constexpr int kSpillProbes = 8;

struct alignas(128) Ctl {
  unsigned long long v;
  unsigned long long pad[15];
};

struct QType {
  float *x, *y, *z, *u, *v, *w, *E;
  uint32_t *vox, *idl, *idh, *hist, *job, *seq;
  Ctl *head, *tail;  // [K]
};

struct QDev {
  QType q[2];  // 0 photons, 1 electrons and positrons
  int K, log2cs;
  uint32_t mask;
  Ctl *next_hist, *idle, *started;
  Ctl *backlog;   // queued particles of each type, all shards (signed; pushes add, claims subtract) [2]
  Ctl *phase;     // 0 source phase, 1 secondary phase
  Ctl *cur_job;   // batch launches: the first job that may still have histories to
                  // start (word 0; word 1 unused)
  Ctl *job_next;  // batch launches: next history of each job [kMaxJobs]
  int refill_min[2];  // idle lanes before a warp refills, by its particle type (photon, electron)
  uint32_t guard[2];               // per-shard bound for sources, by beam type
  long long phase_high[2], phase_low[2];  // global backlog thresholds, by beam type
  uint32_t limit;  // pushes beyond this occupancy of a shard spill over (fault injection can lower it)
  unsigned long long timeout_ns;   // bound on any single wait
  unsigned long long deadline_ns;  // bound on the whole launch (from kernel start)
  uint64_t batch_size;
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// Slot sequence words: the producer publishes a record and the consumer
// frees its slot with a release store; both wait for the word with acquire
// loads, so the record's plain loads and stores are ordered around them.
__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Occupancy of a shard from two relaxed loads.  The loads of head and tail
// may be observed in either order, so a concurrent consumer can make head
// appear ahead of tail: the difference saturates at zero.
__device__ __forceinline__ unsigned long long occupancy(unsigned long long head, unsigned long long tail) {
  return tail > head ? tail - head : 0ull;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lane-level sink: tally with run-length coalescing, counters, and queue
// pushes.  kMulti: a batch launch, whose particles carry their job index.
// kCount: also count events (steps, flights, interactions, tally atomics,
// pushes) for the run statistics; the energy counters (emitted, escaped,
// missed) are always kept.  The event counts live in registers across the
// whole loop and cost about 10 % of the transport rate, so runs count them
// only on request (dpm_run_opts.count_events).  kSauter_: compile in the
// photoelectron angle option (DPM_SAUTER); its code alone, unused, measured
// 4-6 % slower, so only the single-run launches that ask for it carry it.
template <bool kMulti, bool kCount, bool kSauter_ = false>
struct QSink {
  static constexpr bool kSauter = kSauter_;
  const RunParams &R;
  const QDev &Q;
  int home;
  unsigned long long *slab = nullptr;
  int pend_v = -1;
  long long pend_q = 0;
  long long cnt[C_N];
  int err = 0;

  __device__ QSink(const RunParams &r, const QDev &q, int h) : R(r), Q(q), home(h) {
#pragma unroll
    for (int i = 0; i < C_N; ++i) cnt[i] = 0;
  }
  __device__ __forceinline__ static long long fx(float e) { return __float2ll_rn(e * 4294967296.0f); }
  // energy counters (coarser quantum, see kCounterScale)
  __device__ __forceinline__ static long long fxc(float e) { return __float2ll_rn(e * kCounterScaleF); }
  __device__ __forceinline__ void flush() {
    if (pend_v >= 0 && pend_q != 0) {
      atomicAdd(slab + pend_v, (unsigned long long)pend_q);
      if (kCount) ++cnt[C_ATOM];
    }
    pend_v = -1;
    pend_q = 0;
  }
  __device__ __forceinline__ void deposit(int v, float dE) {
    const long long q = fx(dE);
    if (v == pend_v) {
      pend_q += q;
    } else {
      flush();
      pend_v = v;
      pend_q = q;
    }
  }
  __device__ __forceinline__ void escape(float E) { cnt[C_ESC] += fxc(E); }
  __device__ __forceinline__ void error(int e) { err |= e; }
  __device__ __forceinline__ void count_step() {
    if (kCount) ++cnt[C_ESTEP];
  }
  __device__ __forceinline__ void count_flight() {
    if (kCount) ++cnt[C_GFLIGHT];
  }
  __device__ __forceinline__ void count_interaction() {
    if (kCount) ++cnt[C_GINT];
  }

  // Warp-aggregated push of the lanes that are here together: one atomic on
  // the shard's tail per queue type, then each lane writes its record and
  // publishes its slot.
  __device__ DPM_COLD void push(const Part &q) {
    if (kCount) ++cnt[C_PUSH];
    const int t = (q.type == PHOTON) ? 0 : 1;
    const unsigned act = __activemask();
    const unsigned mt = __ballot_sync(act, t == 1);
    // one round per queue type; the masks are the same in every active lane
    for (int tt = 0; tt < 2; ++tt) {
      const unsigned mask = tt ? mt : (act & ~mt);
      if (mask == 0 || t != tt) continue;
      push_one(q, tt, mask);
    }
  }

  __device__ void push_one(const Part &q, int t, unsigned mask) {
    const int leader = __ffs(mask) - 1;
    const int rank = __popc(mask & lanemask_lt());
    const QType &Qt = Q.q[t];
    unsigned long long base = 0;
    int shard = -1;
    if ((int)(threadIdx.x & 31) == leader) {
      // the CTA's own shard, else the next ones (a full shard spills over)
      for (int k = 0; k <= kSpillProbes && k < Q.K; ++k) {
        const int s = (home + k) % Q.K;
        const unsigned long long h = ld_volatile(&Qt.head[s].v);
        const unsigned long long tl = ld_volatile(&Qt.tail[s].v);
        if (occupancy(h, tl) + __popc(mask) <= Q.limit) {
          base = atomicAdd(&Qt.tail[s].v, (unsigned long long)__popc(mask));
          atomicAdd(&Q.backlog[t].v, (unsigned long long)__popc(mask));
          shard = s;
          break;
        }
      }
    }
    base = __shfl_sync(mask, base, leader);
    shard = __shfl_sync(mask, shard, leader);
    if (shard < 0) {
      err |= ERR_OVERFLOW;
      cnt[C_ESC] += fxc(q.E + (q.type == POSITRON ? 2.f * kMc2f : 0.f));
      return;
    }
    const unsigned long long p = base + rank;
    const uint32_t slot = uint32_t(p) & Q.mask;
    const size_t idx = (size_t(shard) << Q.log2cs) + slot;
    // wait for the consumer of position p - capacity to have freed the slot
    if (ld_acquire32(Qt.seq + idx) != uint32_t(p)) {
      const unsigned long long t0 = now_ns();
      while (ld_acquire32(Qt.seq + idx) != uint32_t(p)) {
        if (now_ns() - t0 > Q.timeout_ns) {
          err |= ERR_TIMEOUT;
          return;
        }
        __nanosleep(64);
      }
    }
    Qt.x[idx] = q.x;
    Qt.y[idx] = q.y;
    Qt.z[idx] = q.z;
    Qt.u[idx] = q.u;
    Qt.v[idx] = q.v;
    Qt.w[idx] = q.w;
    Qt.E[idx] = q.E;
    Qt.vox[idx] = uint32_t(q.ix) | (uint32_t(q.iy) << 11) | (uint32_t(q.iz) << 22);
    Qt.idl[idx] = q.id_lo;
    Qt.idh[idx] = q.id_hi;
    Qt.hist[idx] = q.hist | (q.type == POSITRON ? 0x80000000u : 0u);
    if (kMulti) Qt.job[idx] = uint32_t(q.job);
    st_release32(Qt.seq + idx, uint32_t(p + 1));
  }
};

// Leader claims up to `want` queued positions of shard s with a CAS on its
// head; returns the count (warp-uniform) and the first position.
__device__ __forceinline__ int claim(const QType &Qt, int s, int want, unsigned long long &base) {
  int n = 0;
  unsigned long long b = 0;
  if ((threadIdx.x & 31) == 0) {
    for (int tries = 0; tries < 32; ++tries) {
      const unsigned long long h = ld_volatile(&Qt.head[s].v);
      const unsigned long long t = ld_volatile(&Qt.tail[s].v);
      if (t <= h) break;
      const unsigned long long k = min(t - h, (unsigned long long)want);
      if (atomicCAS(&Qt.head[s].v, h, h + k) == h) {
        n = int(k);
        b = h;
        break;
      }
    }
  }
  n = __shfl_sync(kFull, n, 0);
  base = __shfl_sync(kFull, b, 0);
  return n;
}

// Read the record at position p of shard s (waiting for its publication) and
// free the slot for the producer one lap later.
template <bool kMulti>
__device__ __forceinline__ bool take(const QDev &Q, int t, int s, unsigned long long p, Part &o, int &err) {
  const QType &Qt = Q.q[t];
  const uint32_t slot = uint32_t(p) & Q.mask;
  const size_t idx = (size_t(s) << Q.log2cs) + slot;
  if (ld_acquire32(Qt.seq + idx) != uint32_t(p + 1)) {
    const unsigned long long t0 = now_ns();
    while (ld_acquire32(Qt.seq + idx) != uint32_t(p + 1)) {
      if (now_ns() - t0 > Q.timeout_ns) {
        err |= ERR_TIMEOUT;
        return false;
      }
      __nanosleep(32);
    }
  }
  o.x = __ldcg(Qt.x + idx);
  o.y = __ldcg(Qt.y + idx);
  o.z = __ldcg(Qt.z + idx);
  o.u = __ldcg(Qt.u + idx);
  o.v = __ldcg(Qt.v + idx);
  o.w = __ldcg(Qt.w + idx);
  o.E = __ldcg(Qt.E + idx);
  const uint32_t vx = __ldcg(Qt.vox + idx);
  o.ix = int(vx & 0x7ffu);
  o.iy = int((vx >> 11) & 0x7ffu);
  o.iz = int(vx >> 22);
  o.id_lo = __ldcg(Qt.idl + idx);
  o.id_hi = __ldcg(Qt.idh + idx);
  const uint32_t h = __ldcg(Qt.hist + idx);
  o.hist = h & 0x7fffffffu;
  o.type = t == 0 ? PHOTON : ((h >> 31) ? POSITRON : ELECTRON);
  o.job = kMulti ? int(__ldcg(Qt.job + idx)) : 0;
  o.ctr = 0;
  st_release32(Qt.seq + idx, uint32_t(p + (1ull << Q.log2cs)));
  return true;
}

// Fill the warp's empty lanes from queue t (home shard first, then a few
// others).  Returns the number of lanes filled (warp-uniform).
template <bool kMulti>
__device__ int refill_queue(const QDev &Q, int t, int home, int probes, unsigned empty, Part &p, bool &alive,
                            int &err) {
  const int want = __popc(empty);
  if (want == 0) return 0;
  const int lane = threadIdx.x & 31;
  unsigned long long base;
  int s = home;
  int n = claim(Q.q[t], s, want, base);
  for (int k = 1; n == 0 && k <= probes && k < Q.K; ++k) {
    s = (home + k * 97) % Q.K;
    n = claim(Q.q[t], s, want, base);
  }
  if (n == 0) return 0;
  if (lane == 0) atomicAdd(&Q.backlog[t].v, (unsigned long long)(-(long long)n));
  if (empty & (1u << lane)) {
    const int rank = __popc(empty & lanemask_lt());
    if (rank < n) alive = take<kMulti>(Q, t, s, base + rank, p, err);
  }
  return n;
}

// What a particle step of a batch job reads of its job: the phantom and the
// history numbering.  A shared launch copies these records of all its jobs
// into shared memory at the start (64 bytes each, at most kSharedJobs), so
// that a step reads them from shared memory instead of the job table.
struct JobHot {
  DevPhantom P;
  uint64_t first;
  uint32_t key0, key1;
};

struct JobStepCtx {
  const DevTables &T;
  const DevPhantom &P;
  uint64_t first;
  uint32_t key0, key1;
};

__device__ __forceinline__ JobStepCtx job_step_ctx(const RunParams &R, const JobHot *sj, int j) {
  return JobStepCtx{R.T, sj[j].P, sj[j].first, sj[j].key0, sj[j].key1};
}

// Context of a batch job for the source (the job table lives in global memory).
__device__ __forceinline__ JobCtx job_ctx(const RunParams &R, int j) {
  const DevJob &J = R.jobs[j];
  return JobCtx{R.T, J.P, J.S, J.first, J.key0, J.key1};
}

// Start new source histories in the empty lanes: from the run's range, or
// (batch) from the current job of the batch, job after job, so that one
// job's phantom and tally are hot in L2 at a time.  A warp holding particles
// of one type only starts histories of a job with that beam type.
template <bool kMulti, bool kCount, bool kSauter>
__device__ int refill_source(const RunParams &R, const QDev &Q, unsigned empty, Part &p, bool &alive,
                             QSink<kMulti, kCount, kSauter> &sk, int &type) {
  const int want = __popc(empty);
  if (want == 0) return 0;
  const int lane = threadIdx.x & 31;
  unsigned long long b = ~0ull, n = 0;
  int j = 0, jt = type;
  if (lane == 0) {
    if (!kMulti) {
      n = R.n;
      if (ld_volatile(&Q.next_hist->v) < R.n) b = atomicAdd(&Q.next_hist->v, (unsigned long long)want);
    } else {
      for (int tries = 0; tries <= R.n_jobs; ++tries) {
        j = int(ld_volatile(&Q.cur_job[0].v));
        if (j >= R.n_jobs) break;
        jt = R.jobs[j].S.particle == 0 ? 0 : 1;
        if (type >= 0 && jt != type) break;  // the current job has the other beam type
        n = R.jobs[j].n;
        if (ld_volatile(&Q.job_next[j].v) < n) {
          b = atomicAdd(&Q.job_next[j].v, (unsigned long long)want);
          if (b < n) break;
        }
        atomicCAS(&Q.cur_job[0].v, (unsigned long long)j, (unsigned long long)(j + 1));  // job exhausted
        b = ~0ull;
      }
    }
  }
  b = __shfl_sync(kFull, b, 0);
  n = __shfl_sync(kFull, n, 0);
  j = __shfl_sync(kFull, j, 0);
  jt = __shfl_sync(kFull, jt, 0);
  if (b >= n) return 0;
  type = jt;
  if (empty & (1u << lane)) {
    const unsigned long long hl = b + __popc(empty & lanemask_lt());
    if (hl < n) {
      bool hit;
      if (kMulti) {
        hit = make_primary(p, job_ctx(R, j), uint32_t(hl));
        p.job = j;
      } else {
        hit = make_primary(p, R, uint32_t(hl));
      }
      sk.cnt[C_EMIT] += QSink<kMulti, kCount, kSauter>::fxc(p.E);
      if (!hit) sk.cnt[C_MISS] += QSink<kMulti, kCount, kSauter>::fxc(p.E);
      alive = hit;
    }
  }
  return int(min((unsigned long long)want, n - b));
}

// Any queued particle anywhere, or histories left to start (warp-uniform).
template <bool kMulti>
__device__ bool any_work(const RunParams &R, const QDev &Q) {
  bool w = false;
  for (int s = threadIdx.x & 31; s < Q.K && !w; s += 32)
    for (int t = 0; t < 2; ++t)
      if (occupancy(ld_volatile(&Q.q[t].head[s].v), ld_volatile(&Q.q[t].tail[s].v)) > 0) w = true;
  if ((threadIdx.x & 31) == 0) {
    if (!kMulti && ld_volatile(&Q.next_hist->v) < R.n) w = true;
    if (kMulti && ld_volatile(&Q.cur_job[0].v) < (unsigned long long)R.n_jobs) w = true;
  }
  return __any_sync(kFull, w);
}

// Cheap version of any_work() from the global per-type backlog counters
// (exact once the pushes and claims in flight have landed; used to decide
// whether an idle warp should retry, never to end the run).
template <bool kMulti>
__device__ bool any_work_hint(const RunParams &R, const QDev &Q) {
  bool w = false;
  if ((threadIdx.x & 31) == 0) {
    w = (long long)ld_volatile(&Q.backlog[0].v) > 0 || (long long)ld_volatile(&Q.backlog[1].v) > 0;
    if (!kMulti && ld_volatile(&Q.next_hist->v) < R.n) w = true;
    if (kMulti && ld_volatile(&Q.cur_job[0].v) < (unsigned long long)R.n_jobs) w = true;
  }
  return __shfl_sync(kFull, w, 0);
}

// True while both of the CTA's shards hold at most `bound` particles (warp-uniform).
__device__ bool source_allowed(const QDev &Q, int home, unsigned long long bound) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) {
    for (int t = 0; t < 2; ++t)
      if (occupancy(ld_volatile(&Q.q[t].head[home].v), ld_volatile(&Q.q[t].tail[home].v)) > bound) ok = false;
  }
  return __shfl_sync(kFull, ok, 0);
}

// The grid-wide phase (0 source, 1 secondary) for beam type S, switched
// with hysteresis on the global backlog of the other type by whichever warp
// sees the threshold crossed first (warp-uniform).
__device__ int grid_phase(const QDev &Q, int S, unsigned long long *counters) {
  int ph = 0;
  if ((threadIdx.x & 31) == 0) {
    ph = int(ld_volatile(&Q.phase->v));
    const long long b = (long long)ld_volatile(&Q.backlog[1 - S].v);
    if (ph == 0 && b > Q.phase_high[S]) {
      ph = 1;
      if (atomicExch(&Q.phase->v, 1ull) == 0ull) atomicAdd(counters + C_SWITCH, 1ull);
    } else if (ph == 1 && b < Q.phase_low[S]) {
      ph = 0;
      if (atomicExch(&Q.phase->v, 0ull) == 1ull) atomicAdd(counters + C_SWITCH, 1ull);
    }
  }
  return __shfl_sync(kFull, ph, 0);
}

// Beam type of the batch job being started (the table lists photon beams
// first); once every job has been started, that of the last job
// (warp-uniform).
__device__ __forceinline__ int current_source_type(const RunParams &R, const QDev &Q) {
  int t = 0;
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long j = ld_volatile(&Q.cur_job[0].v);
    t = (j < (unsigned long long)R.n_photon_jobs || R.n_photon_jobs == R.n_jobs) ? 0 : 1;
  }
  return __shfl_sync(kFull, t, 0);
}

// True once every source history of the launch has been started (warp-uniform).
template <bool kMulti>
__device__ __forceinline__ bool source_exhausted(const RunParams &R, const QDev &Q) {
  bool e = false;
  if ((threadIdx.x & 31) == 0)
    e = kMulti ? ld_volatile(&Q.cur_job[0].v) >= (unsigned long long)R.n_jobs : ld_volatile(&Q.next_hist->v) >= R.n;
  return __shfl_sync(kFull, e, 0);
}

__device__ void reduce_counters_q(const long long *cnt, int err, const RunParams &R) {
#pragma unroll
  for (int i = 0; i < C_N; ++i) {
    long long v = cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(R.counters + i, (unsigned long long)v);
  }
  int e = err;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e |= __shfl_down_sync(kFull, e, o);
  if ((threadIdx.x & 31) == 0 && e) atomicOr(R.err, e);
}

// Eight resident blocks per SM caps the kernel at 64 registers per thread:
// 32 warps per SM, the fastest of the register/occupancy trade-offs measured.
#ifndef DPM_QUEUE_MIN_BLOCKS
#define DPM_QUEUE_MIN_BLOCKS 8
#endif
template <bool kMulti, bool kCount, bool kSauter = false, bool kPause = false>
__global__ void __launch_bounds__(kQBlock, DPM_QUEUE_MIN_BLOCKS)
    k_queue(const __grid_constant__ RunParams R, const __grid_constant__ QDev Q) {
  const int lane = threadIdx.x & 31;
  const int home = blockIdx.x % Q.K;
  const int src_type = (R.S.particle == 0) ? 0 : 1;
  const size_t V = size_t(R.P.nx) * R.P.ny * R.P.nz;
  if (lane == 0) atomicAdd(&Q.started->v, 1ull);
  QSink<kMulti, kCount, kSauter> sk(R, Q, home);
  Part p{};
  bool alive = false;
  int nstep = 0;
  int mode = -1;  // warp-uniform: type of the particles in the lanes, -1 when empty
  bool idle = false;
  unsigned long long idle_t0 = 0;
  unsigned sleep_ns = 128;
  unsigned retry_ns = 32;
  const unsigned long long t_start = __shfl_sync(kFull, now_ns(), 0);
  // batch launches: the jobs' step records in shared memory (all threads of
  // the block are here, before any divergent code)
  extern __shared__ JobHot sjobs[];
  if (kMulti) {
    for (int j = threadIdx.x; j < R.n_jobs; j += blockDim.x) {
      const DevJob &J = R.jobs[j];
      sjobs[j] = JobHot{J.P, J.first, J.key0, J.key1};
    }
    __syncthreads();
  }
  int cool = 0;  // warp-uniform (kPause): steps before a warp with particles tries to refill again
  for (;;) {
    unsigned live = __ballot_sync(kFull, alive);
    if (live == 0) mode = -1;
    const unsigned live_before = live;
    if (kPause && live != 0 && cool > 0) {
      --cool;
    } else if (live == 0 || 32 - __popc(live) >= Q.refill_min[mode > 0 ? 1 : 0]) {
      const unsigned empty = ~live;
      const bool was_alive = alive;
      const int S = kMulti ? current_source_type(R, Q) : src_type;
      // Source phase: warps start histories and track particles of the
      // beam's type while the secondaries of the other type pile up in
      // the queues; secondary phase: no history starts and warps track the
      // queued particles in full warps.  Warps of the type out of phase
      // finish their lanes and turn over.  A grid-wide phase keeps the SMs
      // on one of the two code paths at a time.
      const int O = 1 - S;
      const int ph = grid_phase(Q, S, R.counters);
      if (mode < 0) {
        if (ph == 1) {
          if (refill_queue<kMulti>(Q, O, home, 0, empty, p, alive, sk.err)) mode = O;
          else if (refill_queue<kMulti>(Q, O, home, kStealProbes, empty, p, alive, sk.err)) mode = O;
          else if (refill_queue<kMulti>(Q, S, home, 0, empty, p, alive, sk.err)) mode = S;
          else if (refill_queue<kMulti>(Q, S, home, kStealProbes, empty, p, alive, sk.err)) mode = S;
        } else {
          int ty = S;
          if (refill_queue<kMulti>(Q, S, home, 0, empty, p, alive, sk.err)) mode = S;
          else if (source_allowed(Q, home, Q.guard[S]) && refill_source<kMulti, kCount, kSauter>(R, Q, empty, p, alive, sk, ty)) mode = S;
          else if (refill_queue<kMulti>(Q, O, home, 0, empty, p, alive, sk.err)) mode = O;
          else if (refill_queue<kMulti>(Q, O, home, kStealProbes, empty, p, alive, sk.err)) mode = O;
          else if (refill_queue<kMulti>(Q, S, home, kStealProbes, empty, p, alive, sk.err)) mode = S;
        }
      } else if (mode == S) {
        int ty = S;
        if (ph == 0 && !refill_queue<kMulti>(Q, S, home, 0, empty, p, alive, sk.err) && source_allowed(Q, home, Q.guard[S]))
          refill_source<kMulti, kCount, kSauter>(R, Q, empty, p, alive, sk, ty);
      } else if (ph == 1 || source_exhausted<kMulti>(R, Q)) {
        refill_queue<kMulti>(Q, O, home, kStealProbes, empty, p, alive, sk.err);
      }
      if (alive && !was_alive) {
        if (kMulti) {
          const DevJob &J = R.jobs[p.job];
          sk.slab = J.slabs + (uint64_t(p.hist) / J.batch_size) * J.V;
        } else {
          sk.slab = R.slabs + (uint64_t(p.hist) / Q.batch_size) * V;
        }
        nstep = 0;
      }
      live = __ballot_sync(kFull, alive);
      if (live != 0u) {
        retry_ns = 32;
        sleep_ns = 128;
      }
      if (kPause) cool = (live != 0u && live == live_before) ? DPM_REFILL_COOLDOWN : 0;
    }
    if (live == 0) {
      // nothing in the lanes: idle until work appears or the run is over
      if (!idle) {
        __threadfence();
        if (lane == 0) atomicAdd(&Q.idle->v, 1ull);
        idle = true;
        idle_t0 = now_ns();
      }
      if (any_work_hint<kMulti>(R, Q)) {
        // work exists but this warp found none within reach: retry after a
        // short, growing pause instead of rescanning at once
        if (lane == 0) atomicAdd(&Q.idle->v, ~0ull);  // -1
        idle = false;
        if (__shfl_sync(kFull, now_ns() - t_start > Q.deadline_ns, 0)) {
          sk.error(ERR_TIMEOUT);
          break;
        }
        __nanosleep(retry_ns);
        retry_ns = min(retry_ns * 2, 2048u);
        continue;
      }
      bool done = false;
      if (lane == 0) done = ld_volatile(&Q.idle->v) == ld_volatile(&Q.started->v);
      done = __shfl_sync(kFull, done, 0);
      if (done) {
        __threadfence();
        if (!any_work<kMulti>(R, Q)) break;
      }
      const bool expired = __shfl_sync(kFull, now_ns() - idle_t0 > Q.timeout_ns, 0);
      if (expired) {
        sk.error(ERR_TIMEOUT);
        break;
      }
      __nanosleep(sleep_ns);
      sleep_ns = min(sleep_ns * 2, 16384u);
      continue;
    }
    if (alive) {
      if (mode == 0) {
        alive = kMulti ? photon_segment(p, job_step_ctx(R, sjobs, p.job), sk, DPM_PHOTON_DRAWS)
                       : photon_segment(p, R, sk, DPM_PHOTON_DRAWS);
        if (alive && ++nstep >= kMaxPhotonSegments * 8) {
          sk.error(ERR_STEPCAP);
          sk.deposit(kMulti ? vox(p, sjobs[p.job].P) : vox(p, R.P), p.E);
          alive = false;
        }
      } else {
        alive = kMulti ? electron_step(p, job_step_ctx(R, sjobs, p.job), sk) : electron_step(p, R, sk);
        if (alive && ++nstep >= kMaxElectronSteps) {
          sk.error(ERR_STEPCAP);
          sk.deposit(kMulti ? vox(p, sjobs[p.job].P) : vox(p, R.P), p.E);
          alive = false;
        }
      }
      if (!alive) sk.flush();
    }
  }
  sk.flush();
  reduce_counters_q(sk.cnt, sk.err, R);
}

__global__ void k_queue_init(uint32_t *seq0, uint32_t *seq1, size_t n, uint32_t mask) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    seq0[i] = uint32_t(i) & mask;
    seq1[i] = uint32_t(i) & mask;
  }
}

}  // namespace

// The queue kernel's instantiations: single run or batch launch (kMulti) x
// event counts x refill pause, and the single runs with the photoelectron
// angle option.
using QKernel = void (*)(RunParams, QDev);
struct QKernelEntry {
  QKernel k;
  bool multi;
};
const QKernelEntry kQueueKernels[10] = {
    {k_queue<false, false>, false},
    {k_queue<false, true>, false},
    {k_queue<true, false>, true},
    {k_queue<true, true>, true},
    {k_queue<false, false, true>, false},
    {k_queue<false, true, true>, false},
    {k_queue<false, false, false, true>, false},
    {k_queue<false, true, false, true>, false},
    {k_queue<true, false, false, true>, true},
    {k_queue<true, true, false, true>, true}};

QKernel queue_kernel(bool multi, bool count, bool sauter, bool pause) {
  if (sauter) return count ? k_queue<false, true, true> : k_queue<false, false, true>;
  if (multi) {
    if (pause) return count ? k_queue<true, true, false, true> : k_queue<true, false, false, true>;
    return count ? k_queue<true, true> : k_queue<true, false>;
  }
  if (pause) return count ? k_queue<false, true, false, true> : k_queue<false, false, false, true>;
  return count ? k_queue<false, true> : k_queue<false, false>;
}

int queue_blocks_per_sm() {
  // single runs keep no shared memory: the whole carveout goes to L1, where
  // the tables are cached; a batch launch keeps its jobs' step records there
  // (kSharedJobs x 64 bytes per block: 8 blocks with their reserved 1 KB
  // each need the 64 KB configuration, 28 % of the 228 KB)
  int best = 1 << 30;
  for (const QKernelEntry &e : kQueueKernels) {
    const QKernel k = e.k;
    int per_sm = 0;
    const bool multi = e.multi;
    const size_t smem = multi ? kSharedJobs * sizeof(JobHot) : 0;
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, multi ? 28 : 0);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kQBlock, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = std::min(best, per_sm);
  }
  return best;
}

int queue_preload() {
  // cudaFuncGetAttributes loads a kernel under lazy module loading
  cudaFuncAttributes a;
  bool ok = cudaFuncGetAttributes(&a, k_queue_init) == cudaSuccess;
  for (const QKernelEntry &e : kQueueKernels) ok = ok && cudaFuncGetAttributes(&a, e.k) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return 0;
  }
  return queue_blocks_per_sm();
}

constexpr int kWordsPerSlot = 13;  // x y z u v w E, voxel, id lo, id hi, history, job, sequence
constexpr int kCtlWords = 8 + kMaxJobs;  // next_hist idle started cur_job[2] backlog[2] phase, job_next[kMaxJobs]

size_t queue_bytes(int K, int log2cs) {
  const size_t slots = size_t(K) << log2cs;
  const size_t per_type = slots * kWordsPerSlot * sizeof(uint32_t) + 2 * size_t(K) * sizeof(Ctl);
  return 2 * per_type + kCtlWords * sizeof(Ctl) + 128;
}

int queue_launch(void *mem, int K, int log2cs, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o,
                 int sm_count, cudaStream_t st, cudaEvent_t start, std::string &err) {
  if (R.jobs && (R.T.flags & DPM_SAUTER)) {
    err = "the photoelectron angle option (DPM_SAUTER) runs in single runs only";
    return DPM_EINVAL;
  }
  if (R.jobs && (R.n_jobs < 1 || R.n_jobs > kSharedJobs)) {
    err = "a shared launch takes 1 to kSharedJobs jobs";
    return DPM_EINVAL;
  }
  const size_t cs = size_t(1) << log2cs;
  const size_t slots = size_t(K) * cs;
  const size_t per_type = slots * kWordsPerSlot * sizeof(uint32_t) + 2 * size_t(K) * sizeof(Ctl);
  QDev Q{};
  char *m = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(mem) + 127) & ~uintptr_t(127));
  Q.next_hist = reinterpret_cast<Ctl *>(m);
  Q.idle = Q.next_hist + 1;
  Q.started = Q.next_hist + 2;
  Q.cur_job = Q.next_hist + 3;  // two words
  Q.backlog = Q.next_hist + 5;  // two words
  Q.phase = Q.next_hist + 7;
  Q.job_next = Q.next_hist + 8;
  char *ctl_end = m + kCtlWords * sizeof(Ctl);
  for (int t = 0; t < 2; ++t) {
    QType &T = Q.q[t];
    char *b = ctl_end + t * per_type;
    T.head = reinterpret_cast<Ctl *>(b);
    T.tail = T.head + K;
    uint32_t *f = reinterpret_cast<uint32_t *>(b + 2 * size_t(K) * sizeof(Ctl));
    float **fl[7] = {&T.x, &T.y, &T.z, &T.u, &T.v, &T.w, &T.E};
    for (int i = 0; i < 7; ++i) *fl[i] = reinterpret_cast<float *>(f + i * slots);
    T.vox = f + 7 * slots;
    T.idl = f + 8 * slots;
    T.idh = f + 9 * slots;
    T.hist = f + 10 * slots;
    T.job = f + 11 * slots;
    T.seq = f + 12 * slots;
  }
  Q.K = K;
  Q.log2cs = log2cs;
  Q.mask = uint32_t(cs - 1);
  Q.refill_min[0] = o.refill_min > 0 ? std::min(o.refill_min, 32) : DPM_REFILL_MIN_G;
  Q.refill_min[1] = o.refill_min > 0 ? std::min(o.refill_min, 32) : DPM_REFILL_MIN_E;
  Q.guard[0] = uint32_t(cs >> DPM_PHASE_GUARD_SHIFT_G);
  Q.guard[1] = uint32_t(cs >> DPM_PHASE_GUARD_SHIFT_E);
  Q.phase_high[0] = (long long)K * (long long)(cs >> DPM_PHASE_HIGH_SHIFT_G);
  Q.phase_low[0] = (long long)K * (long long)(cs >> DPM_PHASE_LOW_SHIFT_G);
  Q.phase_high[1] = (long long)K * (long long)(cs >> DPM_PHASE_HIGH_SHIFT_E);
  Q.phase_low[1] = (long long)K * (long long)(cs >> DPM_PHASE_LOW_SHIFT_E);
  Q.limit = uint32_t(cs - 64);
  if (o.queue_limit > 0) Q.limit = std::min<uint32_t>(Q.limit, uint32_t(o.queue_limit));
  const double tmo = o.timeout_s > 0 ? o.timeout_s : 20.0;
  Q.timeout_ns = (unsigned long long)(tmo * 1e9);
  // the whole launch: the wait bound plus 2 us per history (a hundred times the
  // cost of a 20 MeV electron history on this path)
  Q.deadline_ns = Q.timeout_ns + (unsigned long long)(double(R.n) * 2000.0);
  Q.batch_size = batch_size;
  // zero the control words of both types and the run counters
  const int n_ctl = R.jobs ? 8 + R.n_jobs : 8;
  cudaError_t e = cudaMemsetAsync(m, 0, n_ctl * sizeof(Ctl), st);
  for (int t = 0; t < 2 && e == cudaSuccess; ++t) e = cudaMemsetAsync(Q.q[t].head, 0, 2 * size_t(K) * sizeof(Ctl), st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return DPM_ECUDA;
  }
  k_queue_init<<<sm_count * 4, 256, 0, st>>>(Q.q[0].seq, Q.q[1].seq, slots, Q.mask);
  if (start) cudaEventRecord(start, st);
  const bool count = o.count_events != 0;
  const bool sauter = (R.T.flags & DPM_SAUTER) != 0;
  bool pause = o.refill_pause > 0;
  if (o.refill_pause == 0) {
    // single run: from its own histories (callers on queues below
    // 2^kPauseMinLog2 slots pass -1); a batch launch's caller decides
    const double w = R.S.particle == 0 ? 1.0 : kElectronHistoryWeight;
    pause = !R.jobs && double(R.n) * w <= kPauseMaxHistories;
  }
  const size_t smem = R.jobs ? size_t(R.n_jobs) * sizeof(JobHot) : 0;
  queue_kernel(R.jobs != nullptr, count, sauter, pause)<<<K, kQBlock, smem, st>>>(R, Q);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return DPM_ECUDA;
  }
  return DPM_OK;
}

// Default shard capacity: 2^14 slots; 2^15 for a single electron-beam run,
// whose secondary (photon) phase then starts later and runs longer (20 MeV
// electrons +2 % on the slab phantom, +1.5 % on the 128^3 blobs; 6 MV photons
// -0.3 %, so photon beams keep 2^14).
int default_queue_log2(const RunParams &R) { return (!R.jobs && R.S.particle == 1) ? 15 : 14; }

int queue_prepare(QueueState &q, const dpm_run_opts &o, int sm_count, int &K, int &log2cs, std::string &err) {
  const int per_sm = queue_blocks_per_sm();
  if (per_sm < 1) {
    err = "occupancy query failed";
    return DPM_ECUDA;
  }
  const int bps = o.blocks_per_sm > 0 ? std::min(o.blocks_per_sm, per_sm) : per_sm;
  K = sm_count * bps;
  log2cs = o.queue_log2 > 0 ? o.queue_log2 : 14;
  if (log2cs < 7 || log2cs > 20) {
    err = "queue_log2 must be in [7, 20]";
    return DPM_EINVAL;
  }
  const size_t bytes = queue_bytes(K, log2cs);
  if (q.bytes < bytes) {
    if (q.budget && q.in_use && *q.in_use - q.bytes + bytes > q.budget) {
      err = "device-memory budget of the context exceeded by the particle queues (" + std::to_string(bytes) +
            " bytes)";
      return DPM_ENOMEM;
    }
    if (q.mem) cudaFree(q.mem);
    if (q.in_use) *q.in_use -= q.bytes;
    q.mem = nullptr;
    q.bytes = 0;
    cudaError_t e = cudaMalloc(&q.mem, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      err = std::string("queue allocation: ") + cudaGetErrorString(e);
      return DPM_ENOMEM;
    }
    q.bytes = bytes;
    if (q.in_use) *q.in_use += bytes;
  }
  q.log2_cap = log2cs;
  return DPM_OK;
}

int queue_run(QueueState &q, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o, int sm_count,
              cudaStream_t st, cudaEvent_t start, std::string &err) {
  if (R.n > 0x7fffffffull) {
    err = "the queue kernel takes at most 2^31-1 histories per call";
    return DPM_EINVAL;
  }
  if (R.jobs && (R.n_jobs < 1 || R.n_jobs > kSharedJobs)) {
    err = "bad job count";
    return DPM_EINVAL;
  }
  int K = 0, log2cs = 0;
  dpm_run_opts oq = o;
  if (oq.queue_log2 <= 0) oq.queue_log2 = default_queue_log2(R);
  const int rc = queue_prepare(q, oq, sm_count, K, log2cs, err);
  if (rc) return rc;
  return queue_launch(q.mem, K, log2cs, R, batch_size, o, sm_count, st, start, err);
}

void queue_free(QueueState &q) {
  if (q.mem) cudaFree(q.mem);
  if (q.in_use) *q.in_use -= q.bytes;
  q.mem = nullptr;
  q.bytes = 0;
}

}  // namespace dpm
