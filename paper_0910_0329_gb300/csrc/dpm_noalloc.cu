// dpm_noalloc.cu -- dpm_run_noalloc(): the persistent queue transport for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a host program
// whose device memory is owned by a pool or arena that forbids further device
// allocation, a process working inside a fixed device-memory budget set at
// start-up, or a pipeline that must not add allocation latency or failure
// points to a dose request.  This entry point serves them: it runs the same
// queue kernel as dpm_run() with the same physics and random numbers, but its
// scratch (particle queues, run counters, error word) is a fixed file-scope
// device array, and the integer tally goes straight into a device buffer the
// caller owns.  It calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "dpm_ctx.h"
#include "dpm_internal.h"
#include "dpm_queue.h"

namespace dpm {
namespace {

// Scratch of dpm_run_noalloc(): particle queues plus a 256-byte header
// (run counters and the error word).  The driver places it in a device's
// memory when it loads this file's module there; noalloc_setup() makes that
// happen in dpm_create(), and the array stays until the process exits.
constexpr size_t kNoAllocBytes = size_t(DPM_NOALLOC_SCRATCH_BYTES);
constexpr size_t kHeader = 256;
constexpr int kNoAllocLog2Slots = 9;  // 512 slots per queue shard

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code g_noalloc_scratch is only a host-side stand-in: the device
// address is looked up with the device current.  The lookup is repeated on
// every call (it is cheap once the module is loaded), so that a new primary
// context on the device never leaves a stale address behind.
int scratch_address(void **out, std::string &err) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return DPM_ECUDA;
  }
  *out = p;
  return DPM_OK;
}

}  // namespace

// Called by dpm_create() with the context's device current: loads this
// module (placing the scratch array in device memory) and the queue kernels,
// so that later dpm_run_noalloc() calls find everything resident.
int noalloc_setup(std::string &err) {
  void *p = nullptr;
  const int rc = scratch_address(&p, err);
  if (rc) return rc;
  if (queue_preload() < 1) {
    err = "queue kernel load failed";
    return DPM_ECUDA;
  }
  return DPM_OK;
}

}  // namespace dpm

using namespace dpm;

extern "C" int dpm_run_noalloc(dpm_ctx *c, int phantom_id, const dpm_source *src, uint64_t first_history,
                               uint64_t n_histories, uint64_t seed, int64_t *d_tally, dpm_run_stats *stats) {
  if (!c) return DPM_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  PhantomState *p = ctx_phantom(c, phantom_id);
  if (!p) return ctx_fail(c, DPM_EINVAL, "bad phantom id");
  if (!d_tally) return ctx_fail(c, DPM_EINVAL, "null tally");
  if (n_histories > 0x7fffffffull) return ctx_fail(c, DPM_EINVAL, "at most 2^31-1 histories per call");
  RunParams R{};
  int rc = ctx_run_params(c, p, src, first_history, n_histories, seed, 0, R);
  if (rc) return rc;
  if (n_histories == 0) return DPM_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return ctx_fail(c, DPM_ECUDA, "cudaSetDevice failed");

  void *base = nullptr;
  std::string err;
  if ((rc = scratch_address(&base, err))) return ctx_fail(c, rc, err);

  // shards that fit in the scratch, at most one per resident block
  const int per_sm = queue_blocks_per_sm();
  if (per_sm < 1) return ctx_fail(c, DPM_ECUDA, "occupancy query failed");
  int K = c->sm_count * per_sm;
  while (K > 1 && kHeader + queue_bytes(K, kNoAllocLog2Slots) > kNoAllocBytes) --K;
  if (kHeader + queue_bytes(K, kNoAllocLog2Slots) > kNoAllocBytes)
    return ctx_fail(c, DPM_ENOMEM, "scratch too small for one queue shard");

  // the header holds the run counters and the error word; both start at zero
  unsigned char *hdr = static_cast<unsigned char *>(base);
  if (cudaMemsetAsync(hdr, 0, kHeader, c->stream) != cudaSuccess) return ctx_fail(c, DPM_ECUDA, "memset failed");
  R.n_batches = 1;
  R.slabs = reinterpret_cast<unsigned long long *>(d_tally);  // one batch: the caller's tally
  R.counters = reinterpret_cast<unsigned long long *>(hdr);
  R.err = reinterpret_cast<int *>(hdr + 128);
  dpm_run_opts o{};
  o.count_events = stats ? 1 : 0;
  o.refill_pause = -1;  // 512-slot shards need every refill (kPauseMinLog2)
  if ((rc = queue_launch(hdr + kHeader, K, kNoAllocLog2Slots, R, n_histories, o, c->sm_count, c->stream, nullptr,
                         err)))
    return ctx_fail(c, rc, err);

  // wait, then report the device-side status and counters of this call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return ctx_fail(c, DPM_ECUDA, std::string("transport failed: ") + cudaGetErrorString(e));
  }
  unsigned long long cnt[kCounterSlots];
  int dev_err = 0;
  if (cudaMemcpy(cnt, hdr, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&dev_err, hdr + 128, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, DPM_ECUDA, "status read failed");
  if (stats) {
    stats->n_histories = n_histories;
    stats->n_batches = 1;
    stats->error_flags = dev_err;
    stats->emitted = double((long long)cnt[C_EMIT]) / kCounterScale;
    stats->escaped = double((long long)cnt[C_ESC]) / kCounterScale;
    stats->missed = double((long long)cnt[C_MISS]) / kCounterScale;
    stats->deposited = std::nan("");  // the tally is the caller's: deposited = its increase * 2^-32 MeV
    stats->n_e_steps = cnt[C_ESTEP];
    stats->n_g_flights = cnt[C_GFLIGHT];
    stats->n_g_interactions = cnt[C_GINT];
    stats->n_tally_atomics = cnt[C_ATOM];
    stats->n_pushed = cnt[C_PUSH];
    stats->n_transport_launches = 1;
    stats->n_phase_switches = cnt[C_SWITCH];
  }
  if (dev_err & ERR_OVERFLOW) return ctx_fail(c, DPM_EQUEUE_OVERFLOW, "particle queue overflow in the fixed scratch");
  if (dev_err & ERR_TIMEOUT) return ctx_fail(c, DPM_ETIMEOUT, "a bounded device wait timed out");
  if (dev_err & ERR_STEPCAP) return ctx_fail(c, DPM_ESTEPCAP, "a particle exceeded the step limit");
  return DPM_OK;
}
